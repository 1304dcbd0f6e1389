"""saq_encode_noalloc: the encode for callers that may not allocate device
memory at encode time (a framework that owns all device memory through its
own allocator, a latency-bound ingest thread where an allocation could block
and synchronise the device, a host process that forbids driver allocations
inside its callbacks).  Its scratch is a fixed array inside the library.

The test calls the entry point through the C ABI twice in a row, on two
different batches, and compares each result with saq_encode's on the same
batch.  It builds its own model, so it passes alone in a fresh process as
well as after the other tests; it lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(model, X, codes, factors):
    lib = P.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.saq_encode_noalloc(model.handle, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                  ctypes.c_void_p(codes.data_ptr()),
                                  ctypes.c_void_p(factors.data_ptr()), stream)


def test_noalloc_matches_encode_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    d = 960
    train = synth.power_law(20000, d, 0.8, device="cuda")
    model = P.saq_fit(train, avg_bits=4.0, rounds=6)
    batches = [synth.power_law(3000, d, 0.8, seed=101, device="cuda"),
               synth.power_law(2500, d, 0.8, seed=202, device="cuda")]
    for X in batches:
        n = X.shape[0]
        ref_codes, ref_factors = model.encode(X)
        codes = torch.full((n, model.code_bytes), 0xAB, dtype=torch.uint8, device="cuda")
        factors = torch.full((n, model.factor_count), float("nan"), device="cuda")
        rc = _call_noalloc(model, X, codes, factors)
        assert rc == 0, P.load().saq_last_error()
        torch.cuda.synchronize()
        assert torch.equal(codes, ref_codes)
        assert np.allclose(factors.cpu().numpy(), ref_factors.cpu().numpy(), rtol=1e-6, atol=0)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch.cuda.set_device(0)
    d = 960
    model = P.saq_fit(synth.power_law(5000, d, 0.8, device="cuda"), avg_bits=4.0)
    assert model.d_kept == 960
    nseg = sum(1 for _, _, b in model.plan if b > 0)
    # 32 MiB holds 5 bytes per row and kept dimension plus 4 per row and kept
    # segment, rows in groups of 32
    per_row = 5 * model.d_kept + 4 * nseg
    most = (32 << 20) // (per_row * 32) * 32
    X = synth.power_law(most + 1, d, 0.8, seed=303, device="cuda")
    codes, factors = model.alloc_outputs(most + 1)
    rc = _call_noalloc(model, X, codes, factors)
    assert rc == 1
    msg = P.load().saq_last_error()
    assert b"exceeds the no-allocation scratch" in msg
    assert ("at most %d rows" % most).encode() in msg
    rc = _call_noalloc(model, X[:most], codes[:most], factors[:most])
    assert rc == 0, P.load().saq_last_error()
    ref_codes, ref_factors = model.encode(X[:most].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(codes[:most, :model.code_bytes], ref_codes)
