"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (bars in tests/parity_check.py)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2509_12086_gb300 as P
from paper_2509_12086_gb300 import synth
from tests.parity_check import DIST_TOL, check_codes, gpu_codes_by_round

pytestmark = pytest.mark.gpu


def lib_model(mo, precision="fp32", rounds=6):
    return P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, rounds=rounds,
                              precision=precision)


def precisions():
    return ["fp32_simt", "fp32"]


def check_encode(mo, m, X, rounds=6, label="", **kw):
    """Encode host rows X with model m on the GPU and check the result
    against the oracle's encode of the same rows."""
    eo = O.encode(X, mo, rounds=rounds)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    codes, factors = m.encode(Xd)
    after = lambda: gpu_codes_by_round(m, mo, lambda: m.encode(Xd)[0].cpu().numpy(), rounds)
    return check_codes(mo, eo, codes.cpu().numpy(), factors.cpu().numpy(),
                       O_rows=O.project(X, mo)[0], after=after, rounds=rounds, label=label, **kw)


@pytest.fixture(scope="module")
def c1():
    w = synth.WORKLOADS["c1_d128"]
    X = synth.power_law(w["n"], w["d"], w["alpha"]).numpy()
    Qm = synth.queries(w["nq"], w["d"], w["alpha"]).numpy()
    mo = O.fit(X, w["avg_bits"])
    eo = O.encode(X, mo, rounds=w["rounds"])
    return X, Qm, mo, eo


@pytest.mark.parametrize("prec", precisions())
def test_c1_encode_parity(c1, prec):
    X, Qm, mo, eo = c1
    check_encode(mo, lib_model(mo, prec), X, label="c1_d128 %s" % prec)


def test_c1_quantize_only_parity(c1):
    """Quantize + adjust + pack alone, fed the oracle's projection rounded to
    FP32; the oracle runs on the same rounded values.  Only FP32 rounding in
    the decisions separates the two."""
    X, Qm, mo, _ = c1
    Oo, n2 = O.project(X, mo)
    O32 = Oo.astype(np.float32)
    eo = O.encode_projected(O32.astype(np.float64), n2, mo, rounds=6)
    m = lib_model(mo)
    Od = torch.from_numpy(O32).cuda()
    nd = torch.from_numpy(n2.astype(np.float32)).cuda()
    codes, factors = m.quantize_projected(Od, nd)
    after = lambda: gpu_codes_by_round(m, mo, lambda: m.quantize_projected(Od, nd)[0].cpu().numpy(), 6)
    check_codes(mo, eo, codes.cpu().numpy(), factors.cpu().numpy(), O_rows=O32.astype(np.float64),
                after=after, agree_min=0.9999, margin=1e-6, label="c1_d128 quantize-only")


def test_c1_estimator_parity(c1):
    X, Qm, mo, eo = c1
    m = lib_model(mo)
    # library estimator on the oracle's codes: FP32 arithmetic only
    codes_o = torch.from_numpy(O.pack(eo.codes, mo)).cuda()
    fac_o = torch.from_numpy(eo.factors.astype(np.float32)).cuda()
    Qt = torch.from_numpy(Qm).cuda()
    dl = m.estimate_dist(codes_o, fac_o, Qt).cpu().numpy().astype(np.float64)
    do = O.estimate(mo, eo.codes, eo.factors, Qm)
    assert np.max(np.abs(dl - do) / np.abs(do).max()) < 1e-5
    # end to end: GPU codes and GPU estimator vs oracle codes and estimator
    codes, factors = m.encode(torch.from_numpy(X).cuda())
    dg = m.estimate_dist(codes, factors, Qt).cpu().numpy().astype(np.float64)
    ex = O.exact_dist(X, Qm)
    rg = O.relative_error(dg, ex).mean()
    ro = O.relative_error(do, ex).mean()
    assert abs(rg - ro) <= DIST_TOL, (rg, ro)
    # progressive prefixes (Sec. 3.2)
    for b in (1, 2, 3):
        dlb = m.estimate_dist(codes_o, fac_o, Qt, prefix_bits=b).cpu().numpy()
        dob = O.estimate(mo, eo.codes, eo.factors, Qm, prefix_bits=b)
        assert np.max(np.abs(dlb - dob) / np.abs(dob).max()) < 1e-5


def _random_model(d, plan, seed=0):
    rng = np.random.default_rng(seed)
    dk = sum(l for _, l, b in plan if b > 0)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    # an FP32-representable mean, so that rows equal to it centre to exact zeros
    mean = (rng.standard_normal(d) * 0.1).astype(np.float32).astype(np.float64)
    return O.Model(d=d, mean=mean, W=Q[:dk].copy(), plan=plan)


@pytest.mark.parametrize("prec", precisions())
@pytest.mark.parametrize("n", [1, 13, 1000])
def test_edge_plans_and_ragged_rows(prec, n):
    """Ragged segment (72 coordinates, not a multiple of 32 or 64), a dropped
    segment, B = 1 and B = 8, a 32-wide segment, ragged row counts, and
    rows equal to the mean (all-zero segments)."""
    plan = [(0, 64, 8), (64, 72, 3), (136, 32, 1), (168, 32, 0)]
    mo = _random_model(200, plan)
    rng = np.random.default_rng(n)
    X = (rng.standard_normal((n, 200)) * np.linspace(1, 0.1, 200)).astype(np.float32)
    X[:: 5] = mo.mean.astype(np.float32)
    check_encode(mo, lib_model(mo, prec), X, label="edge plans n=%d %s" % (n, prec))


def test_zero_rows_and_empty_call():
    plan = [(0, 64, 4)]
    mo = _random_model(64, plan)
    m = lib_model(mo)
    X = np.tile(mo.mean.astype(np.float32), (9, 1))
    codes, factors = m.encode(torch.from_numpy(X).cuda())
    c = codes.cpu().numpy()
    f = factors.cpu().numpy()
    assert np.all(c == 0) and np.all(f[:, 1] == 0) and np.all(f[:, 2] == 1)
    codes, factors = m.encode(torch.empty((0, 64), device="cuda"))
    assert codes.shape[0] == 0


def test_long_segment_1024():
    plan = [(0, 1024, 3)]
    mo = _random_model(1024, plan, seed=3)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((300, 1024)).astype(np.float32)
    check_encode(mo, lib_model(mo), X, label="one 1024-long segment")


def test_fit_parity():
    """Library fit (GPU FP64 covariance, cuSOLVER) vs oracle fit (numpy):
    same plan, same variances, same mean, and per kept segment the same
    subspace (W_s^T W_s equals V_s V_s^T; the rotation inside a segment is
    random, so the blocks themselves differ)."""
    X = synth.power_law(20000, 128, 1.0).numpy()
    mo = O.fit(X, 4.0)
    m = P.saq_fit(torch.from_numpy(X).cuda(), avg_bits=4.0)
    assert m.plan == mo.plan
    assert np.allclose(m.variances, mo.sig2, rtol=1e-9, atol=1e-15)
    assert np.allclose(m.mean, mo.mean, rtol=0, atol=1e-12)
    W = m.matrix
    assert np.max(np.abs(W @ W.T - np.eye(W.shape[0]))) < 1e-10
    off = 0
    for (s, l, b) in mo.plan:
        if b == 0:
            continue
        P1 = W[off:off + l].T @ W[off:off + l]
        P2 = mo.W[off:off + l].T @ mo.W[off:off + l]
        assert np.max(np.abs(P1 - P2)) < 1e-8
        off += l


def test_export_import_and_host_path(c1):
    X, Qm, mo, eo = c1
    m = lib_model(mo)
    blob = m.export()
    m2 = P.saq_model_import(blob)
    assert m2.plan == mo.plan and np.array_equal(m2.matrix, mo.W)
    Xd = torch.from_numpy(X).cuda()
    c1_, f1 = m.encode(Xd)
    c2_, f2 = m2.encode(Xd)
    assert torch.equal(c1_, c2_) and torch.equal(f1, f2)
    ch, fh = m.encode_host(torch.from_numpy(X).pin_memory())
    assert np.array_equal(ch.numpy(), c1_.cpu().numpy())
    assert np.array_equal(fh.numpy(), f1.cpu().numpy())


def test_c2_full_size_sampled_rows():
    """d = 960, 4 bits/dim, 1,000,000 rows encoded in the benchmark's launch
    configuration; 20,000 seeded sample rows and the distances of 10,000
    queries to 1,000 of them are checked against the oracle."""
    w = synth.WORKLOADS["c2_d960"]
    n, d = w["n"], w["d"]
    X = synth.power_law(n, d, w["alpha"], device="cuda")
    fit_rows = X[:50000].cpu().numpy()
    mo = O.fit(fit_rows, w["avg_bits"])
    m = lib_model(mo, "fp32")
    codes, factors = m.encode(X)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(7).choice(n, 20000, replace=False))
    it = torch.from_numpy(idx).cuda()
    Xs = X[it].cpu().numpy()
    eo = O.encode(Xs, mo, rounds=w["rounds"])
    Xsd = X[it].contiguous()
    after = lambda: gpu_codes_by_round(m, mo, lambda: m.encode(Xsd)[0].cpu().numpy(), w["rounds"])
    check_codes(mo, eo, codes[it].cpu().numpy(), factors[it].cpu().numpy(),
                O_rows=O.project(Xs, mo)[0], after=after, rounds=w["rounds"],
                label="c2_d960 fp32 (20,000 of 1,000,000 rows)")
    Qm = synth.queries(10000, d, w["alpha"]).numpy()
    sub = idx[:1000]
    ex = O.exact_dist(Xs[:1000], Qm)
    do = O.estimate(mo, eo.codes[:1000], eo.factors[:1000], Qm)
    dg = m.estimate_dist(codes[torch.from_numpy(sub).cuda()], factors[torch.from_numpy(sub).cuda()],
                         torch.from_numpy(Qm).cuda()).cpu().numpy().astype(np.float64)
    assert abs(O.relative_error(dg, ex).mean() - O.relative_error(do, ex).mean()) <= DIST_TOL


@pytest.mark.parametrize("prec,tol", [("fp32_simt", 5e-6), ("fp32", 5e-6), ("bf16", 5e-3),
                                      ("fp8", 5e-2)])
def test_projection_accuracy(c1, prec, tol):
    """saq_project against the oracle's FP64 projection, error relative to the
    row norm |x - c|: FP32 (CUDA cores, or the FP16-split tensor-core GEMM) at
    FP32 rounding level, BF16 and FP8 at their operand rounding."""
    X, Qm, mo, eo = c1
    m = lib_model(mo, prec)
    assert m.tensor_cores == (prec != "fp32_simt")
    Ol, n2 = m.project(torch.from_numpy(X).cuda())
    m.check_device()
    Oo, n2o = O.project(X, mo)
    rel = np.abs(Ol.cpu().numpy().astype(np.float64) - Oo) / np.sqrt(n2o)[:, None]
    assert rel.max() <= tol, rel.max()
    assert np.allclose(n2.cpu().numpy(), n2o, rtol=1e-5)


@pytest.mark.parametrize("n,d,plan", [
    (1, 128, [(0, 64, 5), (64, 64, 3)]),
    (300, 200, [(0, 64, 8), (64, 72, 3), (136, 32, 1), (168, 32, 0)]),
    (1000, 960, [(0, 64, 8), (64, 192, 5), (256, 256, 4), (512, 448, 3)]),
])
def test_tensor_core_projection_ragged(n, d, plan):
    """Ragged rows (not a multiple of the 128-row tile), ragged K (d = 200 is
    not a multiple of the 64-wide K block) and ragged columns (d_kept = 168)."""
    mo = _random_model(d, plan, seed=d)
    rng = np.random.default_rng(n)
    X = (rng.standard_normal((n, d)) * np.linspace(1, 0.05, d)).astype(np.float32)
    m = lib_model(mo, "fp32")
    assert m.tensor_cores
    Ol, n2 = m.project(torch.from_numpy(X).cuda())
    m.check_device()
    Oo, n2o = O.project(X, mo)
    rel = np.abs(Ol.cpu().numpy().astype(np.float64) - Oo) / np.sqrt(n2o)[:, None]
    assert rel.max() <= 5e-6


@pytest.mark.parametrize("prec,u", [("bf16", 2.0 ** -8), ("fp8", 2.0 ** -4)])
@pytest.mark.parametrize("n,d,plan", [
    (1, 128, [(0, 64, 5), (64, 64, 3)]),
    (300, 200, [(0, 64, 8), (64, 72, 3), (136, 32, 1), (168, 32, 0)]),
    (1000, 960, [(0, 64, 8), (64, 192, 5), (256, 256, 4), (512, 448, 3)]),
])
def test_precision_form_projection_ragged(prec, u, n, d, plan):
    """The BF16 / FP8 projection (A operand in TMEM) on ragged rows, a ragged
    K tail (d = 200 pads to 224 for BF16's 32-value K blocks, to 256 for FP8's
    64) and ragged columns, against the FP64 projection.  Rounding both
    operands to a format of unit roundoff u (BF16 2^-8, E4M3 2^-4; the scales
    are powers of two) bounds each output by |o_i - o~_i| <= (2u + u^2)
    sum_k |w_ik| |y_k| <= (2u + u^2) |w_i| |y| with |w_i| = 1 (orthonormal
    rows of W) and y = x - c.  The interleaved layout the encode uses holds
    the same values."""
    mo = _random_model(d, plan, seed=d)
    rng = np.random.default_rng(n + d)
    X = (rng.standard_normal((n, d)) * np.linspace(1, 0.05, d)).astype(np.float32)
    m = lib_model(mo, prec)
    assert m.tensor_cores
    Xd = torch.from_numpy(X).cuda()
    Ol, _ = m.project(Xd)
    Oi, _ = m.project_interleaved(Xd)
    m.check_device()
    Oo, n2o = O.project(X, mo)
    rel = np.abs(Ol.cpu().numpy().astype(np.float64) - Oo) / np.sqrt(n2o)[:, None]
    bound = 2 * u + u * u
    assert rel.max() <= bound * 1.001, (rel.max(), bound)
    # typical errors sit far below the worst case (a misplaced operand gives O(1))
    assert rel.mean() <= bound / 8, (rel.mean(), bound)
    dk = mo.d_kept
    g = (n + 31) // 32
    Ore = Oi.view(g, dk, 32).permute(0, 2, 1).reshape(g * 32, dk)[:n]
    assert torch.equal(Ore, Ol)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_precision_forms_error_bounded(c1, prec):
    """BF16 / FP8 projection (quantization and adjustment stay FP32): codes
    differ from the oracle's where the projection error crosses a decision,
    so only the error statistics are bounded.  The projection adds its own
    error energy: rounding both operands to unit roundoff u (BF16 2^-8, E4M3
    2^-4; uniform rounding errors of variance u^2/3 each) gives about
    2u^2/3 = 1e-5 (BF16) or 2.6e-3 (FP8) of |x - c|^2, so the
    mean quantization error may exceed the oracle's by 10% (BF16) or by an
    absolute 0.01 (FP8, 4x the budget); the estimator error stays within 2x
    (BF16) or 4x (FP8) of the oracle's."""
    X, Qm, mo, eo = c1
    m = lib_model(mo, prec)
    codes, factors = m.encode(torch.from_numpy(X).cuda())
    f = factors.cpu().numpy().astype(np.float64)
    eg, eo_ = O.quant_error(f, mo).mean(), O.quant_error(eo.factors, mo).mean()
    lim = 0.10 * eo_ if prec == "bf16" else 0.01
    assert abs(eg - eo_) <= lim, (eg, eo_)
    dg = m.estimate_dist(codes, factors, torch.from_numpy(Qm).cuda()).cpu().numpy()
    ex = O.exact_dist(X, Qm)
    rg = O.relative_error(dg.astype(np.float64), ex).mean()
    ro = O.relative_error(O.estimate(mo, eo.codes, eo.factors, Qm), ex).mean()
    assert rg <= (2.0 if prec == "bf16" else 4.0) * ro + 1e-4, (rg, ro)


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_interleaved_halves_equal_encode(c1, prec):
    """saq_project_ex + saq_quantize_projected_ex in the encode's own layout
    (rows in groups of 32) reproduce saq_encode bit for bit, including a
    ragged last group."""
    X, Qm, mo, eo = c1
    m = lib_model(mo, prec)
    Xd = torch.from_numpy(X[:9999]).cuda()
    ref_c, ref_f = m.encode(Xd)
    Oi, nrm = m.project_interleaved(Xd)
    c, f = m.quantize_interleaved(Oi, nrm)
    assert torch.equal(c, ref_c) and torch.equal(f, ref_f)


def test_c1_staged_estimator_parity(c1):
    """Sec. 4.3 multi-stage bounds: the library on the oracle's codes against
    the oracle (FP32 arithmetic only), the last stage against the library's
    own estimate, the basis through export/import and through saq_fit, and
    the error for a model without a basis."""
    X, Qm, mo, eo = c1
    m = P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, basis=O.kept_basis(mo))
    assert m.has_basis
    codes_o = torch.from_numpy(O.pack(eo.codes, mo)).cuda()
    fac_o = torch.from_numpy(eo.factors.astype(np.float32)).cuda()
    Qt = torch.from_numpy(Qm).cuda()
    k = len(mo.kept)
    for mc in (0.0, 1.0, 3.0):
        bl = m.estimate_staged(codes_o, fac_o, Qt, mc).cpu().numpy().astype(np.float64)
        bo = O.estimate_staged(mo, eo.codes, eo.factors, Qm, mc)
        assert bl.shape == bo.shape == (Qm.shape[0], X.shape[0], k + 1)
        assert np.max(np.abs(bl - bo)) / np.abs(bo).max() < 1e-5, mc
    dl = m.estimate_dist(codes_o, fac_o, Qt).cpu().numpy()
    assert np.max(np.abs(bl[:, :, k] - dl)) / np.abs(dl).max() < 1e-6
    m2 = P.saq_model_import(m.export())
    assert m2.has_basis
    b2 = m2.estimate_staged(codes_o, fac_o, Qt, 3.0).cpu().numpy()
    assert np.array_equal(b2, bl.astype(np.float32))
    # saq_fit records the basis; its last stage is its own estimate
    mf = P.saq_fit(torch.from_numpy(X).cuda(), avg_bits=4.0)
    assert mf.has_basis
    cf, ff = mf.encode(torch.from_numpy(X).cuda())
    bf = mf.estimate_staged(cf, ff, Qt, 2.0).cpu().numpy()
    df = mf.estimate_dist(cf, ff, Qt).cpu().numpy()
    assert np.max(np.abs(bf[:, :, -1] - df)) / np.abs(df).max() < 1e-6
    # without a basis the bounds are unavailable
    m0 = lib_model(mo)
    assert not m0.has_basis
    with pytest.raises(P.SaqError):
        m0.estimate_staged(codes_o, fac_o, Qt, 2.0)


def test_host_path_several_chunks_equals_device_encode():
    """saq_encode_host stages about 128 MB of rows per chunk in three slots:
    at d = 4096 that is 8,192 rows, so 100,000 rows run twelve full chunks
    and a partial one and reuse every slot; every output must equal the
    device encode of the same rows."""
    torch.cuda.set_device(0)
    d = 4096
    X = synth.power_law(100_000, d, 0.6, device="cuda")
    m = P.saq_fit(X[:20000].contiguous(), avg_bits=2.0)
    cd, fd = m.encode(X)
    Xh = X.cpu().pin_memory()
    ch, fh = m.encode_host(Xh)
    torch.cuda.synchronize()
    assert torch.equal(ch, cd.cpu())
    assert torch.equal(fh, fd.cpu())


@pytest.mark.parametrize("d", [6144, 6400])
def test_largest_dimensions(d):
    """d = 6144 is the largest dimension the tensor-core projection takes
    (the centring term of a whole row sits in shared memory beside the
    stages).  Beyond it a tensor-core precision is refused with
    SAQ_ERR_UNSUPPORTED, explicitly (no silent switch of the projection),
    and the CUDA-core projection (fp32_simt) must be chosen; both encodes
    agree with the oracle."""
    plan = [(0, 1024, 4), (1024, 2048, 2), (3072, d - 3072, 1)]
    mo = _random_model(d, plan, seed=d)
    rng = np.random.default_rng(d)
    X = (rng.standard_normal((300, d)) * np.linspace(1, 0.05, d)).astype(np.float32)
    if d > 6144:
        with pytest.raises(P.SaqError, match="unsupported"):
            lib_model(mo, "fp32")
        m = lib_model(mo, "fp32_simt")
        assert not m.tensor_cores
        with pytest.raises(P.SaqError, match="unsupported"):
            m.set_precision("bf16")
        assert not m.tensor_cores  # a refused precision leaves the model as it was
    else:
        m = lib_model(mo, "fp32")
        assert m.tensor_cores
    check_encode(mo, m, X, label="d=%d" % d)
    m.check_device()


def test_more_kept_segments_than_supported_is_an_error():
    """The quantize kernel takes at most 64 kept segments per model; a plan
    with more is refused with an error, not encoded."""
    d = 65 * 16
    plan = [(i * 16, 16, 2) for i in range(65)]
    mo = _random_model(d, plan, seed=3)
    m = lib_model(mo, "fp32")
    X = torch.randn(64, d, device="cuda")
    with pytest.raises(P.SaqError):
        m.encode(X)


@pytest.mark.parametrize("prec", precisions())
def test_odd_segment_lengths(prec):
    """Segments of 5, 13, 70, 37 and 3 coordinates at offsets that are no
    multiple of 8: the partial batches of the initial pass, the rounds and
    the packing, a segment spanning two 64-bit words, and projection blocks
    that straddle segment ends."""
    plan = [(0, 5, 4), (5, 13, 6), (18, 70, 3), (88, 37, 2), (125, 3, 1)]
    mo = _random_model(128, plan, seed=5)
    rng = np.random.default_rng(17)
    X = (rng.standard_normal((1000, 128)) * np.linspace(1, 0.1, 128)).astype(np.float32)
    check_encode(mo, lib_model(mo, prec), X, label="odd segment lengths %s" % prec)
