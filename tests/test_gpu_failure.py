"""Failure detection on the GPU without a GPU fault.

The tensor-core projection bounds every pipeline wait; a wait that reaches
its bound raises the device error flag, every role leaves its loop, the
copies and MMAs in flight are drained, tensor memory is freed and the kernel
returns.  Here the bound is set to 1 ns (saq_set_wait_limit), so that the
waits run out on their own, and the tests check that the status comes back
(SAQ_ERR_TIMEOUT from saq_check_device, from the synchronous host-buffer
encode and from the ingest service) and that the next normal encode meets
parity.  Rows outside the operand format's range (FP32 split) or not finite
(any form) come back as SAQ_ERR_RANGE.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth
from tests.test_gpu_parity import check_encode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch.cuda.set_device(0)
    X = synth.power_law(6000, 256, 0.8).numpy()
    mo = O.fit(X, 4.0)
    return X, mo


def _model(mo, precision="fp32"):
    return P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, rounds=6,
                              precision=precision)


def test_wait_timeout_is_reported_and_the_next_encode_is_correct(setup):
    X, mo = setup
    m = _model(mo)
    Xd = torch.from_numpy(X).cuda()
    Xh = torch.from_numpy(X).pin_memory()
    m.encode(Xd)
    m.check_device()  # a normal encode leaves no flag
    P.saq_set_wait_limit(1)
    try:
        m.encode(Xd)  # asynchronous: the status comes from the check
        with pytest.raises(P.SaqError, match="timed out"):
            m.check_device()
        with pytest.raises(P.SaqError, match="timed out"):
            m.encode_host(Xh)  # synchronous: reports the timeout itself
    finally:
        P.saq_set_wait_limit(0)
    m.check_device()  # the flag was cleared by the reports
    check_encode(mo, m, X, label="after a timed-out launch")


def test_out_of_range_row_is_reported(setup):
    X, mo = setup
    m = _model(mo)
    Xb = X[:500].copy()
    # about 10^4 times a typical row: scaled coordinates beyond FP16's 65504
    Xb[7] = (Xb[7] - mo.mean) * 1e4 + mo.mean
    Xd = torch.from_numpy(Xb).cuda()
    m.encode(Xd)
    with pytest.raises(P.SaqError, match="out of range"):
        m.check_device()
    with pytest.raises(P.SaqError, match="out of range"):
        m.encode_host(torch.from_numpy(Xb).pin_memory())
    # a row 100 times a typical one is within range and encodes normally
    Xb[7] = (X[7] - mo.mean) * 100 + mo.mean
    check_encode(mo, m, Xb, label="a row 100x a typical one")
    m.check_device()
    # a non-finite row is reported in the BF16 form too
    mb = _model(mo, "bf16")
    Xn = X[:300].copy()
    Xn[3, 5] = np.nan
    mb.encode(torch.from_numpy(Xn).cuda())
    with pytest.raises(P.SaqError, match="out of range"):
        mb.check_device()
    mb.encode(torch.from_numpy(X[:300].copy()).cuda())
    mb.check_device()


def test_ingest_reports_a_timed_out_batch_and_recovers(setup):
    X, mo = setup
    m = _model(mo)
    svc = P.Ingest([m], hbm_budget_bytes=1 << 30, max_batch_rows=2048, slots=2)
    try:
        Xh = torch.from_numpy(X[:3000].copy()).pin_memory()
        P.saq_set_wait_limit(1)
        try:
            t = svc.submit(0, Xh)
            with pytest.raises(P.SaqError, match="timed out"):
                svc.wait(t, timeout_ms=60000)
        finally:
            P.saq_set_wait_limit(0)
        t = svc.submit(0, Xh)
        codes, factors, _ = svc.wait(t, timeout_ms=60000)
        rc, rf = m.encode(Xh.cuda())
        assert np.array_equal(codes.numpy(), rc.cpu().numpy())
        assert np.array_equal(factors.numpy(), rf.cpu().numpy())
    finally:
        svc.close()
    m.check_device()
