"""The larger configurations at full size, checked against the oracle on
seeded sample rows: d = 1536 at 2 bits/dim (FP32 strict parity, BF16
precision form) and d = 3072 at 1 and 8 bits/dim (FP8 precision form).

The oracle fits its own model on a 40,000-row subsample; the library imports
it, encodes every row in the launch configuration of the benchmark, and the
sampled rows are compared.  The FP32 path meets the strict parity bars of
tests/parity_check.py (every code mismatch traced to an oracle near-tie).
The precision forms' error against the oracle (code agreement, quantization
error, relative distance error) is printed per configuration (pytest -s,
lines starting "PRECISION") and bounded by the operand-rounding budgets
derived in test_gpu_parity.py::test_precision_forms_error_bounded.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth
from tests.parity_check import check_codes, gpu_codes_by_round

pytestmark = pytest.mark.gpu


def _run(n, d, alpha, bits, precisions, sample=4000, queries=300):
    X = synth.power_law(n, d, alpha, device="cuda")
    mo = O.fit(X[:40000].cpu().numpy(), bits)
    idx = np.sort(np.random.default_rng(11).choice(n, sample, replace=False))
    it = torch.from_numpy(idx).cuda()
    Xs = X[it].cpu().numpy()
    eo = O.encode(Xs, mo, rounds=6)
    Os = O.project(Xs, mo)[0]
    Qm = synth.queries(queries, d, alpha).numpy()
    ex = O.exact_dist(Xs[:1000], Qm)
    ro = O.relative_error(O.estimate(mo, eo.codes[:1000], eo.factors[:1000], Qm), ex).mean()
    eps_o = O.quant_error(eo.factors, mo).mean()
    out = {}
    for prec in precisions:
        m = P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, rounds=6, precision=prec)
        codes, factors = m.encode(X)
        m.check_device()
        cs = codes[it].cpu().numpy()
        fs = factors[it].cpu().numpy()
        agree = float((O.unpack(cs, mo) == eo.codes).mean())
        eps_v = O.quant_error(fs.astype(np.float64), mo)
        eps = eps_v.mean()
        de = np.abs(eps_v - O.quant_error(eo.factors, mo))
        sub = torch.from_numpy(idx[:1000]).cuda()
        dg = m.estimate_dist(codes[sub], factors[sub], torch.from_numpy(Qm).cuda()).cpu().numpy()
        rg = O.relative_error(dg.astype(np.float64), ex).mean()
        Xsd = X[it].contiguous()
        after = (lambda m=m, Xsd=Xsd: gpu_codes_by_round(
            m, mo, lambda: m.encode(Xsd)[0].cpu().numpy(), 6))
        out[prec] = dict(agree=agree, eps=eps, eps_oracle=eps_o, rel_err=rg, rel_err_oracle=ro,
                         codes=cs, factors=fs, O_rows=Os, after=after)
        print("PRECISION d=%d bits=%.0f %s: code agreement %.5f, mean eps %.4e (oracle %.4e), "
              "mean |eps diff| %.3e, max |eps diff| %.3e, mean rel. distance error %.4e "
              "(oracle %.4e)" % (d, bits, prec, agree, eps, eps_o, de.mean(), de.max(), rg, ro))
        del codes, factors
    return mo, eo, out


def test_d1536_2bits_fp32_and_bf16():
    mo, eo, out = _run(1_000_000, 1536, 0.6, 2.0, ["fp32", "bf16"])
    r = out["fp32"]
    check_codes(mo, eo, r["codes"], r["factors"], O_rows=r["O_rows"], after=r["after"],
                label="c3_d1536 2 b/dim fp32")
    assert abs(r["rel_err"] - r["rel_err_oracle"]) <= 1e-4
    b = out["bf16"]
    assert abs(b["eps"] - b["eps_oracle"]) <= 0.10 * b["eps_oracle"]
    assert b["rel_err"] <= 2.0 * b["rel_err_oracle"] + 1e-4


@pytest.mark.parametrize("bits", [1.0, 8.0])
def test_d3072_fp8(bits):
    mo, eo, out = _run(500_000, 3072, 0.5, bits, ["fp8", "fp32"], sample=2000)
    r = out["fp32"]
    check_codes(mo, eo, r["codes"], r["factors"], O_rows=r["O_rows"], after=r["after"],
                label="c4_d3072 %.0f b/dim fp32" % bits)
    f = out["fp8"]
    # E4M3 operand rounding adds about 2.6e-3 of |x - c|^2 (4x budget: 0.01)
    assert abs(f["eps"] - f["eps_oracle"]) <= 0.01
    assert f["rel_err"] <= 4.0 * f["rel_err_oracle"] + 2e-3
