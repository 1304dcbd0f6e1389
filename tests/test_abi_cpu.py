"""The C-ABI library without a GPU: it loads, exports every symbol the header
declares, its host-side plan search agrees with the oracle, and argument
checks fail before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "saq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(saq_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = P.load()
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(_lib.EXPORTS) == syms


def test_params_defaults():
    p = _lib.saq_params()
    P.load().saq_params_init(ctypes.byref(p))
    assert (p.avg_bits, p.max_bits, p.rounds, p.seg_granularity, p.precision) == (4.0, 8, 6, 64, 0)
    assert p.tie_frac == pytest.approx(1e-3) and p.seed == 4


@pytest.mark.parametrize("d,alpha,avg,g", [
    (128, 1.0, 4.0, 64), (960, 0.8, 4.0, 64), (1536, 0.6, 2.0, 64), (3072, 0.5, 1.0, 64),
    (3072, 0.5, 8.0, 64), (256, 1.2, 0.5, 64), (200, 1.0, 3.0, 64), (16, 1.2, 4.0, 1),
    (100, 0.0, 2.5, 8),
])
def test_library_plan_equals_oracle_plan(d, alpha, avg, g):
    """Algorithm 2 in the library (host C++) and in the oracle (C), written
    separately from the same reading, choose the same plan."""
    sig2 = np.arange(1, d + 1, dtype=np.float64) ** (-alpha)
    quota = int(round(avg * d))
    po = O.plan_dp(sig2, quota, g=g)
    segs, err = P.saq_plan_search(sig2, quota, g=g)
    assert segs == po.segments
    assert err == pytest.approx(po.error, rel=1e-14)


def test_library_plan_on_fitted_spectra():
    rng = np.random.default_rng(0)
    for _ in range(5):
        s2 = np.sort(rng.gamma(0.5, size=192))[::-1].copy()
        po = O.plan_dp(s2, 3 * 192, g=64)
        segs, _ = P.saq_plan_search(s2, 3 * 192, g=64)
        assert segs == po.segments


def test_invalid_arguments_rejected_without_gpu():
    lib = P.load()
    rc = lib.saq_encode(None, None, 10, None, None, None)
    assert rc == 1 and b"NULL" in lib.saq_last_error()
    with pytest.raises(P.SaqError, match="invalid argument"):
        # plan does not cover d
        P.saq_model_create(8, np.zeros(8), np.eye(8)[:4], [(0, 4, 2)])
    with pytest.raises(P.SaqError, match="invalid argument"):
        P.saq_model_create(8, np.zeros(8), np.eye(8), [(0, 8, 9)])
    with pytest.raises(P.SaqError):
        P.saq_plan_search(np.ones(8), -1, g=1)
    with pytest.raises(P.SaqError, match="not a model blob"):
        P.saq_model_import(b"nope" * 10)
