"""Serving form: continuous-batching ingest over three resident collections.

* Each request's result through the service, mixed with the others, equals
  saq_encode of the same rows alone (BF16 and FP32 projection).
* A batch holds pieces of several collections and runs as ONE projection
  launch and ONE quantize launch (the library's launch counter moves by two
  per batch).
* Admission by HBM budget: with a budget that holds little more than one
  batch, the device memory in flight never exceeds it and queued work waits
  for it.
* Served rows of a seeded sample meet the oracle parity bars (FP32) or the
  BF16 operand-rounding bounds.
"""
import re

import numpy as np
import pytest
import torch

import oracle as O
import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth
from tests.parity_check import check_codes, gpu_codes_by_round

pytestmark = pytest.mark.gpu

SPECS = [(128, 4.0), (960, 4.0), (1536, 2.0)]


@pytest.fixture(scope="module")
def collections():
    torch.cuda.set_device(0)
    models, oracle_models = [], []
    for d, bits in SPECS:
        X = synth.power_law(20000, d, 0.8, seed=11 + d)
        mo = O.fit(X.numpy(), bits)
        oracle_models.append(mo)
        models.append(P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, rounds=6))
    return models, oracle_models


def _requests(count, seed, max_rows=9000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        c = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(max_rows))))
        X = synth.power_law(n, SPECS[c][0], 0.8, seed=seed * 1000 + i).pin_memory()
        out.append((c, X))
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_ingest_mix_equals_alone_in_two_launches_per_batch(collections, prec):
    """One slot: whole-batch requests of the d = 1536 collection occupy it
    (about 3 ms each) while a burst of small requests of all three
    collections queues behind them, so that the next batches take pieces of
    several collections in arrival order."""
    models, _ = collections
    for m in models:
        m.set_precision(prec)
    try:
        svc = P.Ingest(models, hbm_budget_bytes=8 << 30, max_batch_rows=65536, slots=1)
        # six whole-batch requests (the same rows, read-only) hold the slot
        # for well over the time the burst takes to submit
        blk = synth.power_law(65536, SPECS[2][0], 0.8, seed=77).pin_memory()
        reqs = [(2, blk)] * 6 + _requests(40, 5)
        l0 = P.saq_kernel_launch_count()
        tickets = [(c, X, svc.submit(c, X)) for c, X in reqs]
        results = [(c, X) + svc.wait(t, timeout_ms=60000) for c, X, t in tickets]
        st = svc.stats()
        launches = P.saq_kernel_launch_count() - l0
        svc.close()
        assert st["completed"] == 46 and st["submitted"] == 46
        assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
        # batches mix collections, and each batch is one projection launch
        # plus one quantize launch over all of its collections
        assert st["mixed_batches"] >= 1
        assert launches == 2 * st["batches"], (launches, st["batches"])
        for c, X, codes, factors, lat in results:
            rc, rf = models[c].encode(X.cuda())
            assert np.array_equal(codes.numpy(), rc.cpu().numpy())
            assert np.array_equal(factors.numpy(), rf.cpu().numpy())
            assert lat > 0
    finally:
        for m in models:
            m.set_precision("fp32")


def test_ingest_admission_by_hbm_budget(collections):
    models, _ = collections
    with pytest.raises(P.SaqError, match="exceed the HBM budget") as e:
        P.Ingest(models, hbm_budget_bytes=1 << 20, max_batch_rows=65536, slots=4)
    with pytest.raises(P.SaqError, match="exceed the HBM budget") as e:
        P.Ingest([models[1]], hbm_budget_bytes=1 << 20, max_batch_rows=65536, slots=4)
    one = int(re.search(r"\((\d+) bytes\)", str(e.value)).group(1))
    # room for one whole batch of the d = 960 collection and a fifth of
    # another: with four slots and four whole-batch requests, work must wait
    # for memory, not for a slot
    budget = one * 6 // 5
    svc = P.Ingest([models[1]], hbm_budget_bytes=budget, max_batch_rows=65536, slots=4)
    reqs = [synth.power_law(65536, SPECS[1][0], 0.8, seed=900 + i).pin_memory() for i in range(4)]
    tickets = [(X, svc.submit(0, X)) for X in reqs]
    results = [(X,) + svc.wait(t, timeout_ms=120000) for X, t in tickets]
    st = svc.stats()
    svc.close()
    assert 0 < st["peak_bytes_in_flight"] <= budget
    assert st["deferred_batches"] > 0
    assert st["batches"] >= 5  # a batch that the budget cut short
    for X, codes, factors, _ in results:
        rc, rf = models[1].encode(X.cuda())
        assert np.array_equal(codes.numpy(), rc.cpu().numpy())
        assert np.array_equal(factors.numpy(), rf.cpu().numpy())
    # argument errors
    svc = P.Ingest(models, hbm_budget_bytes=1 << 30, max_batch_rows=1024, slots=1)
    with pytest.raises(P.SaqError, match="no collection"):
        svc.submit(7, torch.zeros((3, 128)))
    t = svc.submit(0, torch.zeros((5000, 128)))
    codes, factors, lat = svc.wait(t, timeout_ms=60000)
    assert codes.shape[0] == 5000
    svc.close()


def _plain_model(d, plan, precision, seed):
    rng = np.random.default_rng(seed)
    dk = sum(l for _, l, b in plan if b > 0)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    mean = rng.standard_normal(d) * 0.05
    return P.saq_model_create(d, mean, Q[:dk].copy() if dk else np.zeros((0, d)), plan,
                              rounds=6, precision=precision)


def test_ingest_projection_kinds_share_batches_only_when_compatible():
    """Collections of different projection kinds in one service: FP32 split
    and FP8 tensor-core models, a CUDA-core model (fp32_simt) and a model
    whose plan drops every segment (only |x - c|^2 is stored).  Rows of
    different tensor-core precisions or of the CUDA-core model never share a
    launch; a model without kept dimensions joins any batch.  Every request
    still equals saq_encode of its rows alone."""
    torch.cuda.set_device(0)
    models = [_plain_model(128, [(0, 64, 5), (64, 64, 3)], "fp32", 1),
              _plain_model(256, [(0, 128, 4), (128, 128, 2)], "fp8", 2),
              _plain_model(96, [(0, 64, 4), (64, 32, 2)], "fp32_simt", 3),
              _plain_model(64, [(0, 64, 0)], "fp32", 4),
              _plain_model(192, [(0, 64, 8), (64, 128, 1)], "fp8", 5)]
    assert [m.tensor_cores for m in models] == [True, True, False, False, True]
    assert models[3].d_kept == 0 and models[3].code_bytes == 0
    dims = [m.d for m in models]
    svc = P.Ingest(models, hbm_budget_bytes=4 << 30, max_batch_rows=65536, slots=1)
    rng = np.random.default_rng(8)
    blocker = synth.power_law(65536, 256, 0.8, seed=55).pin_memory()
    reqs = [(1, blocker)] * 16
    for i in range(60):
        c = int(rng.integers(0, len(models)))
        n = int(np.exp(rng.uniform(0, np.log(3000))))
        reqs.append((c, synth.power_law(n, dims[c], 0.8, seed=700 + i).pin_memory()))
    tickets = [(c, X, svc.submit(c, X)) for c, X in reqs]
    results = [(c, X) + svc.wait(t, timeout_ms=60000) for c, X, t in tickets]
    st = svc.stats()
    svc.close()
    assert st["completed"] == len(reqs)
    assert st["mixed_batches"] >= 1
    for c, X, codes, factors, _ in results:
        rc, rf = models[c].encode(X.cuda())
        assert np.array_equal(codes.numpy()[:, :models[c].code_bytes], rc.cpu().numpy())
        assert np.array_equal(factors.numpy(), rf.cpu().numpy())


def test_served_rows_against_the_oracle(collections):
    """A seeded sample of the rows served in a mixed run, per collection,
    against the FP64 oracle: FP32 strict parity (every mismatch traced to an
    oracle near-tie), BF16 within its operand-rounding bounds (mean
    quantization error within 10% of the oracle's)."""
    models, oracle_models = collections
    reqs = _requests(30, 21)
    for prec in ("fp32", "bf16"):
        for m in models:
            m.set_precision(prec)
        svc = P.Ingest(models, hbm_budget_bytes=8 << 30, max_batch_rows=65536, slots=1)
        blk = synth.power_law(65536, SPECS[2][0], 0.8, seed=78).pin_memory()
        blockers = [svc.submit(2, blk) for _ in range(6)]
        tickets = [(c, X, svc.submit(c, X)) for c, X in reqs]
        got = [(c, X) + svc.wait(t, timeout_ms=60000)[:2] for c, X, t in tickets]
        for t in blockers:
            svc.wait(t, timeout_ms=60000)
        assert svc.stats()["mixed_batches"] >= 1
        svc.close()
        rng = np.random.default_rng(3)
        for c in range(3):
            mine = [(X, cd, f) for cc, X, cd, f in got if cc == c]
            if not mine:
                continue
            X = torch.cat([x for x, _, _ in mine]).numpy()
            codes = torch.cat([cd for _, cd, _ in mine]).numpy()
            factors = torch.cat([f for _, _, f in mine]).numpy()
            idx = np.sort(rng.choice(X.shape[0], min(1500, X.shape[0]), replace=False))
            mo, m = oracle_models[c], models[c]
            Xs = np.ascontiguousarray(X[idx])
            eo = O.encode(Xs, mo, rounds=6)
            if prec == "fp32":
                Xd = torch.from_numpy(Xs).cuda()
                after = (lambda m=m, Xd=Xd, mo=mo: gpu_codes_by_round(
                    m, mo, lambda: m.encode(Xd)[0].cpu().numpy(), 6))
                check_codes(mo, eo, np.ascontiguousarray(codes[idx]), factors[idx],
                            O_rows=O.project(Xs, mo)[0], after=after,
                            label="served d=%d fp32" % SPECS[c][0])
            else:
                eg = O.quant_error(factors[idx].astype(np.float64), mo).mean()
                e0 = O.quant_error(eo.factors, mo).mean()
                agree = float((O.unpack(np.ascontiguousarray(codes[idx]), mo) == eo.codes).mean())
                print("SERVED d=%d bf16: code agreement %.5f, mean eps %.4e (oracle %.4e)"
                      % (SPECS[c][0], agree, eg, e0))
                assert abs(eg - e0) <= 0.10 * e0
    for m in models:
        m.set_precision("fp32")
