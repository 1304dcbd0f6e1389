"""Serving form: continuous-batching ingest over three resident collections.
Each request's result through the service, mixed with the others, equals
saq_encode of the same rows alone."""
import numpy as np
import pytest
import torch

import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def collections():
    torch.cuda.set_device(0)
    specs = [(128, 4.0), (960, 4.0), (1536, 2.0)]
    models = []
    for d, bits in specs:
        X = synth.power_law(20000, d, 0.8, seed=11 + d, device="cuda")
        models.append(P.saq_fit(X, avg_bits=bits))
    return specs, models


def test_ingest_mix_equals_alone(collections):
    specs, models = collections
    svc = P.Ingest(models, hbm_budget_bytes=4 << 30, max_batch_rows=4096, slots=3)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(40):
        c = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(9000))))
        X = synth.power_law(n, specs[c][0], 0.8, seed=1000 + i).pin_memory()
        reqs.append((c, X, svc.submit(c, X)))
    for c, X, t in reqs:
        codes, factors, lat = svc.wait(t, timeout_ms=60000)
        rc, rf = models[c].encode(X.cuda())
        assert np.array_equal(codes.numpy(), rc.cpu().numpy())
        assert np.array_equal(factors.numpy(), rf.cpu().numpy())
        assert lat > 0
    st = svc.stats()
    assert st["completed"] == 40 and st["submitted"] == 40
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    assert st["batches"] >= 10
    svc.close()


def test_ingest_admission_and_errors(collections):
    specs, models = collections
    with pytest.raises(P.SaqError, match="exceed the HBM budget"):
        P.Ingest(models, hbm_budget_bytes=1 << 20, max_batch_rows=65536, slots=4)
    svc = P.Ingest(models, hbm_budget_bytes=1 << 30, max_batch_rows=1024, slots=1)
    with pytest.raises(P.SaqError, match="no collection"):
        svc.submit(7, torch.zeros((3, 128)))
    t = svc.submit(0, torch.zeros((5000, 128)))
    codes, factors, lat = svc.wait(t, timeout_ms=60000)
    assert codes.shape[0] == 5000
    svc.close()
