"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a worked
example derived by hand from the paper, brute force on tiny inputs, a closed
form, an invariant, a special case that reduces to a known method, or a bound
the paper prints.  A plausible slip in the oracle (dropped term, wrong sign,
wrong index, swapped operand) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from tests.conftest import golden

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def cos_explicit(u, o):
    """Cosine of Eq. adj-obj computed from scratch (no incremental state)."""
    return float(np.dot(u, o) / (np.linalg.norm(u) * np.linalg.norm(o)))


# ---------------------------------------------------------------- rotations
@pytest.mark.parametrize("n", [1, 2, 7, 64, 200])
def test_haar_rotation_is_orthonormal(n):
    """Random orthonormal matrix (Sec. 2.2, Sec. 4.1): R^T R = I to 1e-12."""
    R = O.haar(n, np.random.default_rng(11))
    assert np.max(np.abs(R.T @ R - np.eye(n))) <= 1e-12
    assert np.max(np.abs(R @ R.T - np.eye(n))) <= 1e-12


def test_haar_rotation_is_not_biased():
    """Haar: over many draws E[R] = 0 and E[R_ij^2] = 1/n (a QR without the
    sign fix has a positive diagonal bias and fails the first check)."""
    rng = np.random.default_rng(5)
    n, k = 4, 4000
    acc = np.zeros((n, n))
    acc2 = np.zeros((n, n))
    for _ in range(k):
        R = O.haar(n, rng)
        acc += R
        acc2 += R * R
    assert np.max(np.abs(acc / k)) < 0.05
    assert np.max(np.abs(acc2 / k - 1.0 / n)) < 0.02


# ---------------------------------------------------------------------- PCA
def _power_law(n, d, alpha, seed=1):
    rng = np.random.default_rng(seed)
    lam = np.arange(1, d + 1, dtype=np.float64) ** (-alpha)
    Q = O.haar(d, np.random.default_rng(seed + 100))
    Z = rng.standard_normal((n, d)) * np.sqrt(lam)
    return Z @ Q.T, lam, Q


def test_pca_eigen_equation_and_spectrum():
    """Sec. 4.1: eigen-pairs of the covariance, sigma^2 descending; the
    eigenvalues match the generator's spectrum within sampling error
    (relative sd of a sample variance ~ sqrt(2/N)); the mean matches 0."""
    n, d = 40000, 24
    X, lam, _ = _power_law(n, d, 1.0)
    c, s2, V = O.pca(X)
    Y = X - c
    C = Y.T @ Y / n
    res = np.max(np.abs(C @ V - V * s2))
    assert res <= 1e-10 * np.max(np.abs(C))
    assert np.all(np.diff(s2) <= 0)
    assert np.max(np.abs(V.T @ V - np.eye(d))) < 1e-12
    assert np.all(np.abs(s2 / lam - 1.0) < 6.0 * math.sqrt(2.0 / n) + 0.02)
    assert np.max(np.abs(c)) < 6.0 / math.sqrt(n)
    # canonical sign: largest-magnitude component positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(d)] > 0)


def test_fit_matrix_rows_orthonormal_and_plan_cover():
    X, _, _ = _power_law(5000, 128, 1.0)
    m = O.fit(X, 4.0)
    assert sum(l for _, l, _ in m.plan) == 128
    starts = [s for s, _, _ in m.plan]
    assert starts == sorted(starts) and starts[0] == 0
    for (s, l, _), (s2, _, _) in zip(m.plan, m.plan[1:]):
        assert s + l == s2
    W = m.W
    assert np.max(np.abs(W @ W.T - np.eye(W.shape[0]))) < 1e-12
    # each kept block spans exactly the PCA eigenvectors of its segment
    c, s2v, V = O.pca(X)
    off = 0
    for (s, l, b) in m.plan:
        if b == 0:
            continue
        Ws = W[off:off + l]
        P1 = Ws.T @ Ws
        P2 = V[:, s:s + l] @ V[:, s:s + l].T
        assert np.max(np.abs(P1 - P2)) < 1e-10
        off += l


# ------------------------------------------------------------ plan (DP)
def _read_plans():
    out = []
    g = golden("plan_worked_examples.txt")
    for key, v in g.items():
        parts = " ".join(v).split("|")
        sig2 = np.array([float(x) for x in parts[0].split()[1:]])
        quota = int(parts[1].split()[1])
        maxb = int(parts[2].split()[1])
        plan = [tuple(int(t) for t in p.split(",")) for p in parts[3].split()[1:]]
        err = float(parts[4].split()[1])
        cost = int(parts[5].split()[1])
        out.append((key, sig2, quota, maxb, plan, err, cost))
    return out


@pytest.mark.parametrize("case", _read_plans(), ids=lambda c: c[0])
def test_plan_worked_examples(case):
    _, sig2, quota, maxb, plan, err, cost = case
    p = O.plan_dp(sig2, quota, g=1, max_bits=maxb)
    assert p.segments == plan
    assert p.error == pytest.approx(err, rel=1e-15)
    assert p.cost == cost


def _brute_force_plans(sig2, g, quota, max_bits):
    """Every plan: all segmentations of the grid and all bit choices."""
    D = len(sig2)
    pos = list(range(0, D, g)) + [D]
    npos = len(pos)
    prefix = np.concatenate([[0.0], np.cumsum(sig2)])
    out = []
    for cut in itertools.product([0, 1], repeat=npos - 2):
        bounds = [0] + [i + 1 for i, c in enumerate(cut) if c] + [npos - 1]
        segs = [(pos[a], pos[b] - pos[a]) for a, b in zip(bounds, bounds[1:])]
        for bits in itertools.product(range(max_bits + 1), repeat=len(segs)):
            costb = sum(b * l for (_, l), b in zip(segs, bits))
            if costb > quota:
                continue
            e = 0.0
            for (s, l), b in zip(segs, bits):
                e = e + math.ldexp(prefix[s + l] - prefix[s], -b)
            out.append((e, len(segs), costb, [(s, l, b) for (s, l), b in zip(segs, bits)]))
    return out


def _select(plans, tie):
    emin = min(p[0] for p in plans)
    band = [p for p in plans if p[0] <= emin * (1 + tie)]
    k = min(p[1] for p in band)
    cand = [p for p in band if p[1] == k]
    e = min(p[0] for p in cand)
    cost = min(p[2] for p in cand if p[0] == e)
    return emin, k, e, cost


@pytest.mark.parametrize("spec", [
    ("powerlaw", 1.0, 4.0), ("powerlaw", 0.6, 2.0), ("powerlaw", 1.5, 1.0),
    ("powerlaw", 0.8, 7.0), ("step", 0.0, 3.0), ("uniform", 0.0, 4.0),
])
def test_plan_matches_brute_force_grid64(spec):
    """Algorithm 2 (with the segment-count rule) equals exhaustive search
    over every segmentation on the 64-grid and every bit choice, D = 320."""
    kind, alpha, avg = spec
    D, g = 320, 64
    if kind == "powerlaw":
        sig2 = np.arange(1, D + 1, dtype=np.float64) ** (-alpha)
    elif kind == "step":
        sig2 = np.where(np.arange(D) < 100, 5.0, 0.1)
    else:
        sig2 = np.ones(D)
    quota = int(round(avg * D))
    p = O.plan_dp(sig2, quota, g=g, max_bits=8, tie_frac=1e-3)
    emin, k, e, cost = _select(_brute_force_plans(sig2, g, quota, 8), 1e-3)
    assert p.min_error == pytest.approx(emin, rel=1e-13)
    assert len(p.segments) == k
    assert p.error == pytest.approx(e, rel=1e-13)
    assert p.cost == cost
    assert O.plan_error(sig2, p.segments) == pytest.approx(p.error, rel=1e-12)


def test_plan_d16_g1_monotone_brute_force():
    """D = 16, g = 1, bits 0..8, average 4 bits.  The modelled error only
    depends on the per-dimension bits; with sigma^2 sorted descending an
    exchange argument makes non-increasing allocations optimal, also for the
    fewest-runs rule, so brute force over all C(24, 8) = 735,471
    non-increasing allocations is exhaustive."""
    D = 16
    sig2 = np.arange(1, D + 1, dtype=np.float64) ** (-1.2)
    quota = 64
    p = O.plan_dp(sig2, quota, g=1, max_bits=8, tie_frac=1e-3)
    allocs = np.array(list(itertools.combinations_with_replacement(range(8, -1, -1), D)),
                      dtype=np.int64)
    cost = allocs.sum(axis=1)
    ok = cost <= quota
    allocs, cost = allocs[ok], cost[ok]
    err = (sig2[None, :] * np.ldexp(1.0, -allocs)).sum(axis=1)
    runs = 1 + (np.diff(allocs, axis=1) != 0).sum(axis=1)
    emin = err.min()
    band = err <= emin * (1 + 1e-3)
    k = runs[band].min()
    sel = band & (runs == k)
    e = err[sel].min()
    assert p.min_error == pytest.approx(emin, rel=1e-12)
    assert len(p.segments) == k
    assert p.error == pytest.approx(e, rel=1e-12)
    bits = [b for _, l, b in p.segments for _ in range(l)]
    assert all(a >= b for a, b in zip(bits, bits[1:]))


def test_plan_uniform_spectrum_single_segment():
    """Sec. 4.2: with a uniform spectrum the plan is one segment at the
    average bit width (SAQ reduces to CAQ)."""
    for D, avg in [(128, 4), (960, 4), (256, 1), (1536, 2)]:
        p = O.plan_dp(np.full(D, 0.37), avg * D, g=64, max_bits=8)
        assert p.segments == [(0, D, avg)]


def test_plan_remainder_segment():
    """g does not divide D: the last segment takes the remainder."""
    sig2 = np.arange(1, 201, dtype=np.float64) ** -1.0
    p = O.plan_dp(sig2, 800, g=64, max_bits=8)
    assert sum(l for _, l, _ in p.segments) == 200
    for s, l, _ in p.segments[:-1]:
        assert l % 64 == 0
    assert p.cost <= 800


# ------------------------------------------------------------- CAQ (Alg. 1)
def test_caq_worked_example():
    g = golden("caq_worked_example.txt")
    o = np.array([float(x) for x in g["o"]])
    B, r = int(g["bits"][0]), int(g["rounds"][0])
    c0, *_ = O.caq_segment(o, B, 0)
    assert c0.tolist() == [int(x) for x in g["init_codes"]]
    c, nrm, cs, acc, mt, mi, ic = O.caq_segment(o, B, r)
    assert c.tolist() == [int(x) for x in g["final_codes"]]
    assert acc.tolist() == [int(x) for x in g["accepts"]]
    assert nrm == pytest.approx(1.05, rel=1e-15)
    assert ic == pytest.approx(float(g["init_cos"][0]), abs=1e-13)
    assert cs == pytest.approx(float(g["final_cos"][0]), abs=1e-13)


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 8])
def test_init_code_is_nearest_midpoint(B):
    """Eq. find_nearest_code: each initial code selects the interval midpoint
    -v_max + Delta (c + 0.5) nearest to o[i] (brute force over 2^B)."""
    rng = np.random.default_rng(B)
    o = rng.standard_normal(97)
    c, *_ = O.caq_segment(o, B, 0)
    v = np.max(np.abs(o))
    delta = 2 * v / 2 ** B
    mids = -v + delta * (np.arange(2 ** B) + 0.5)
    nearest = np.argmin(np.abs(o[:, None] - mids[None, :]), axis=1)
    assert np.array_equal(c, nearest)


def test_b1_reduces_to_sign_code_without_moves():
    """B = 1: all codewords have the same norm, the sign code maximises the
    cosine (RaBitQ's 1-bit code, Sec. 2.2), and Algorithm 1 moves nothing."""
    rng = np.random.default_rng(3)
    for len_ in [64, 128, 448]:
        o = rng.standard_normal(len_)
        c, nrm, cs, acc, *_ = O.caq_segment(o, 1, 6)
        assert np.array_equal(c, (o >= 0).astype(np.uint8))
        assert acc.sum() == 0
        assert cs == pytest.approx(np.sum(np.abs(o)) / (math.sqrt(len_) * nrm), rel=1e-13)


def test_b1_cosine_concentrates_near_0_8():
    """Sec. 2.2: <o_bar, o> of the 1-bit code concentrates around 0.8; for a
    Gaussian direction E|z| / sqrt(E z^2) = sqrt(2/pi) = 0.7979."""
    rng = np.random.default_rng(9)
    vals = [O.caq_segment(rng.standard_normal(512), 1, 0)[2] for _ in range(200)]
    assert abs(np.mean(vals) - math.sqrt(2 / math.pi)) < 0.005
    assert np.std(vals) < 0.02


@pytest.mark.parametrize("B", [2, 3, 4, 6])
def test_rounds_never_lower_cosine(B):
    """Algorithm 1 keeps only strictly improving moves: the cosine after r
    rounds is non-decreasing in r, and rises whenever a round moves."""
    rng = np.random.default_rng(20 + B)
    for _ in range(20):
        o = rng.standard_normal(64) * np.linspace(2.0, 0.5, 64)
        prev = O.caq_segment(o, B, 0)[2]
        for r in range(1, 8):
            c, nrm, cs, acc, *_ = O.caq_segment(o, B, r)
            assert cs >= prev - 1e-15
            if acc[r - 1] > 0:
                assert cs > prev
            prev = cs


@pytest.mark.parametrize("B", [2, 3, 4])
def test_converged_code_is_a_local_optimum(B):
    """After enough rounds, no single +-1 code change raises the cosine
    (checked from scratch), and zero-move rounds repeat forever (early exit
    after a round without a move gives the same result)."""
    rng = np.random.default_rng(40 + B)
    cmax = 2 ** B - 1
    for _ in range(10):
        o = rng.standard_normal(40)
        c, nrm, cs, acc, *_ = O.caq_segment(o, B, 60)
        assert acc[-1] == 0
        first_zero = int(np.argmax(acc == 0))
        assert np.all(acc[first_zero:] == 0)
        c2, _, cs2, *_ = O.caq_segment(o, B, first_zero + 1)
        assert np.array_equal(c, c2) and cs2 == cs
        u = 2.0 * c - cmax
        base = cos_explicit(u, o)
        assert base == pytest.approx(cs, abs=1e-13)
        for i in range(len(o)):
            for dlt in (+1, -1):
                if 0 <= int(c[i]) + dlt <= cmax:
                    u2 = u.copy()
                    u2[i] += 2 * dlt
                    assert cos_explicit(u2, o) <= base + 1e-13


@pytest.mark.parametrize("B,d", [(2, 5), (3, 4), (2, 6)])
def test_caq_between_init_and_brute_force_optimum(B, d):
    """Tiny d: cos(init) <= cos(CAQ) <= max over the whole grid G (brute
    force, Sec. 3.3 codebook), and CAQ gets close to the optimum."""
    rng = np.random.default_rng(100 * B + d)
    grid = np.array(list(itertools.product(range(2 ** B), repeat=d)), dtype=np.float64)
    U = 2 * grid - (2 ** B - 1)
    Un = U / np.linalg.norm(U, axis=1, keepdims=True)
    gaps = []
    for _ in range(30):
        o = rng.standard_normal(d)
        best = np.max(Un @ o) / np.linalg.norm(o)
        c, nrm, cs, acc, mt, mi, ic = O.caq_segment(o, B, 8)
        assert ic <= cs + 1e-15
        assert cs <= best + 1e-12
        gaps.append(best - cs)
    assert np.mean(gaps) < 0.01


def test_error_falls_about_4x_per_bit():
    """Sec. 4.2: relative error of a segment ~ 2^-B on inner products, so the
    squared residual 1 - cos^2 falls about 4x per added bit (d = 128)."""
    rng = np.random.default_rng(17)
    vecs = [rng.standard_normal(128) for _ in range(200)]
    errs = []
    for B in range(1, 9):
        errs.append(np.mean([1 - O.caq_segment(v, B, 6)[2] ** 2 for v in vecs]))
    ratios = [errs[i] / errs[i + 1] for i in range(1, 7)]
    assert all(3.0 <= r <= 5.0 for r in ratios), ratios


def test_zero_segment_reading():
    c, nrm, cs, acc, *_ = O.caq_segment(np.zeros(64), 4, 6)
    assert np.all(c == 0) and nrm == 0 and cs == 1.0 and acc.sum() == 0


# ------------------------------------------------------------ code layout
def test_pack_worked_example_and_prefix():
    g = golden("pack_worked_example.txt")
    L, B = int(g["len"][0]), int(g["bits"][0])
    m = O.Model(d=L, mean=np.zeros(L), W=np.eye(L), plan=[(0, L, B)])
    codes = np.zeros((1, L), dtype=np.uint8)
    head = [int(x) for x in g["codes_head"]]
    codes[0, :len(head)] = head
    packed = O.pack(codes, m)
    assert packed[0].tolist() == [int(x, 16) for x in g["bytes"]]
    assert np.array_equal(O.unpack(packed, m), codes)
    rng = np.random.default_rng(0)
    m2 = O.Model(d=200, mean=np.zeros(200), W=np.eye(200)[:136],
                 plan=[(0, 64, 5), (64, 72, 3), (136, 64, 0)])
    codes = np.concatenate([rng.integers(0, 32, (7, 64)), rng.integers(0, 8, (7, 72))],
                           axis=1).astype(np.uint8)
    pk = O.pack(codes, m2)
    assert pk.shape[1] == m2.code_bytes == 5 * 8 + 3 * 16
    assert np.array_equal(O.unpack(pk, m2), codes)
    # the first b planes of a segment are floor(c / 2^(B-b)) (Sec. 3.2)
    plane0 = np.unpackbits(pk[:, :8], axis=1, bitorder="little")
    assert np.array_equal(plane0, codes[:, :64] >> 4)


# -------------------------------------------------------------- estimator
def _single_segment_model(d, B, seed=7):
    R = O.haar(d, np.random.default_rng(seed))
    return O.Model(d=d, mean=np.zeros(d), W=R, plan=[(0, d, B)])


@pytest.mark.parametrize("B", [2, 4, 6])
def test_estimator_meets_the_printed_error_bound(B):
    """Sec. 2.3 remark: for unit vectors the inner-product error of the
    estimator is below 2^-B * 5.75 / sqrt(D) with > 99.9% probability for the
    optimal code; CAQ is near optimal (Sec. 3.3), so at most 1% of pairs may
    exceed it."""
    d = 256
    rng = np.random.default_rng(B)
    X = rng.standard_normal((200, d))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Qm = rng.standard_normal((50, d))
    Qm /= np.linalg.norm(Qm, axis=1, keepdims=True)
    m = _single_segment_model(d, B)
    e = O.encode(X, m, rounds=8)
    est = O.estimate(m, e.codes, e.factors, Qm)
    ip_est = (1.0 + 1.0 - est) / 2.0
    err = np.abs(ip_est - Qm @ X.T)
    bound = 2.0 ** -B * 5.75 / math.sqrt(d)
    assert np.mean(err > bound) <= 0.01


def test_estimator_unbiased_and_closed_form():
    """Sec. 2.2 lemma / Sec. 3.2: the estimate is linear in q with
    d2_est - d2 = -2 sum_kept <q_s, r_s> + 2 sum_dropped <q_s, o_s>,
    r_s = |o_s| u_s / (|u_s| cos_s) - o_s; over zero-mean queries the mean
    signed error is zero."""
    X, _, _ = _power_law(3000, 128, 1.0, seed=4)
    m = O.fit(X, 2.0)
    e = O.encode(X[:40], m, rounds=6)
    rng = np.random.default_rng(8)
    cov = np.cov(X.T)
    L = np.linalg.cholesky(cov + 1e-12 * np.eye(128))
    Qm = m.mean + rng.standard_normal((4000, 128)) @ L.T
    est = O.estimate(m, e.codes, e.factors, Qm)
    ex = O.exact_dist(X[:40], Qm)
    diff = est - ex
    # unbiased over queries (per data vector, 5 standard errors)
    mu = diff.mean(axis=0)
    se = diff.std(axis=0) / math.sqrt(diff.shape[0])
    assert np.all(np.abs(mu) <= 5 * se + 1e-9)
    # closed form, built from the full orthonormal PCA basis
    c, s2, V = O.pca(X)
    Oproj, _ = O.project(X[:40], m)
    Qc = Qm - m.mean
    Qp, _ = O.project(Qm, m)
    pred = np.zeros_like(diff)
    for j, (off, l, b) in enumerate(m.kept):
        u = 2.0 * e.codes[:, off:off + l] - (2 ** b - 1)
        nr = e.factors[:, 1 + 2 * j]
        cs = e.factors[:, 2 + 2 * j]
        r = nr[:, None] * u / (np.linalg.norm(u, axis=1) * cs)[:, None] - Oproj[:, off:off + l]
        pred += -2.0 * Qp[:, off:off + l] @ r.T
    for (s, l, b) in m.plan:
        if b == 0:
            Vd = V[:, s:s + l]
            pred += 2.0 * (Qc @ Vd) @ ((X[:40] - m.mean) @ Vd).T
    assert np.max(np.abs(pred - diff)) < 1e-9 * np.max(np.abs(ex))


def test_quant_error_matches_explicit_residual():
    """Per-vector error = residual of the best rescaling of o_bar_a per kept
    segment plus the dropped energy, over |x - c|^2."""
    X, _, _ = _power_law(3000, 128, 1.0, seed=6)
    m = O.fit(X, 1.5)
    e = O.encode(X[:30], m, rounds=6)
    Oproj, n2 = O.project(X[:30], m)
    res = n2 - np.sum(Oproj ** 2, axis=1)
    for j, (off, l, b) in enumerate(m.kept):
        o = Oproj[:, off:off + l]
        u = 2.0 * e.codes[:, off:off + l] - (2 ** b - 1)
        a = np.sum(u * o, axis=1) / np.sum(u * u, axis=1)
        res += np.sum((o - a[:, None] * u) ** 2, axis=1)
    assert np.allclose(O.quant_error(e.factors, m), res / n2, rtol=1e-10, atol=1e-14)


def test_progressive_prefix_is_a_valid_estimator():
    """Sec. 3.2: the b-bit prefix with Delta' = Delta 2^(B-b) still estimates
    distances; its error sits between the full code's and the 1-bit code's."""
    X, _, _ = _power_law(4000, 128, 0.5, seed=12)
    m = O.fit(X, 8.0)
    e = O.encode(X[:200], m, rounds=6)
    Qm = X[-100:]
    ex = O.exact_dist(X[:200], Qm)
    full = O.relative_error(O.estimate(m, e.codes, e.factors, Qm), ex).mean()
    p4 = O.relative_error(O.estimate(m, e.codes, e.factors, Qm, prefix_bits=4), ex).mean()
    p1 = O.relative_error(O.estimate(m, e.codes, e.factors, Qm, prefix_bits=1), ex).mean()
    assert full < p4 < p1
    assert p1 < 0.5


def test_progressive_prefix_worked_example():
    """Sec. 3.2: the b-bit prefix floor(c / 2^(B-b)) with Delta' = Delta 2^(B-b)
    and the stored factors reused, against values worked by hand
    (tests/golden/prefix_worked_example.txt).  A wrong grid offset (2^B - 1
    instead of 2^b - 1), a prefix taken from the low bits, or a norm of the
    full code in place of the prefix's fails it."""
    g = golden("prefix_worked_example.txt")
    m = O.Model(d=4, mean=np.zeros(4), W=np.eye(4), plan=[(0, 4, int(g["bits"][0]))])
    codes = np.array([[int(v) for v in g["codes"]]], dtype=np.uint8)
    factors = np.array([[float(v) for v in g["factors"]]])
    q = np.array([[float(v) for v in g["query"]]])
    for b in (3, 2, 1):
        want = float(g["d2_b%d" % b][0])
        got = O.estimate(m, codes, factors, q, prefix_bits=b)[0, 0]
        assert got == pytest.approx(want, rel=1e-14), b
    # prefix_bits >= B (and 0) is the full code
    assert O.estimate(m, codes, factors, q, prefix_bits=5)[0, 0] == pytest.approx(
        float(g["d2_b3"][0]), rel=1e-14)


# ------------------------------------------------- decision trace of Alg. 1
def _state_before(tr, r, i):
    """Codes of the state at which round r (1-based) reaches coordinate i:
    coordinates before i already carry round r's values."""
    c = tr.codes_after[r - 1].astype(np.int64).copy()
    c[:i] = tr.codes_after[r, :i]
    return c


@pytest.mark.parametrize("B", [2, 3, 5])
def test_trace_gaps_are_cosine_differences_from_scratch(B):
    """Each recorded gap equals the change of the cosine of Eq. adj-obj,
    recomputed from scratch (codeword Delta (c + 0.5) - v_max, no running
    state), of moving coordinate i by +-1 from the state the scan is in when
    it reaches i; moves out of [0, 2^B - 1] are -inf."""
    rng = np.random.default_rng(40 + B)
    o = rng.standard_normal(23) * np.linspace(1.5, 0.3, 23)
    rounds = 4
    tr = O.caq_trace(o, B, rounds)
    v = np.max(np.abs(o))
    delta = 2 * v / 2 ** B
    cmax = 2 ** B - 1
    for r in range(1, rounds + 1):
        for i in range(len(o)):
            c = _state_before(tr, r, i)
            base = cos_explicit(delta * (c + 0.5) - v, o)
            for s, rec in ((1, tr.dplus), (-1, tr.dminus)):
                if not 0 <= c[i] + s <= cmax:
                    assert rec[r - 1, i] == -np.inf
                    continue
                cn = c.copy()
                cn[i] += s
                want = cos_explicit(delta * (cn + 0.5) - v, o) - base
                assert rec[r - 1, i] == pytest.approx(want, abs=1e-13)


@pytest.mark.parametrize("B", [2, 4, 6])
def test_trace_decisions_follow_algorithm_1(B):
    """The recorded codes move exactly as Algorithm 1 decides from the
    recorded gaps (+Delta first, kept iff the cosine strictly rises; -Delta
    only if +Delta was not kept), the last row is the plain run's code and
    every row r equals a plain run of r rounds; the per-coordinate initial
    margins are the distances to the nearest interior interval boundary
    (brute force over the 2^B - 1 boundaries of Eq. find_nearest_code)."""
    rng = np.random.default_rng(60 + B)
    o = rng.standard_normal(57) * np.linspace(2.0, 0.2, 57)
    rounds = 5
    tr = O.caq_trace(o, B, rounds)
    for r in range(rounds + 1):
        assert np.array_equal(tr.codes_after[r], O.caq_segment(o, B, r)[0])
    moves = tr.codes_after[1:].astype(int) - tr.codes_after[:-1].astype(int)
    want = np.where(tr.dplus > 0, 1, np.where(tr.dminus > 0, -1, 0))
    assert np.array_equal(moves, want)
    v = np.max(np.abs(o))
    delta = 2 * v / 2 ** B
    bounds = -v + delta * np.arange(1, 2 ** B)
    brute = np.min(np.abs(o[:, None] - bounds[None, :]), axis=1) / np.linalg.norm(o)
    assert np.allclose(tr.init_margin, brute, rtol=1e-12, atol=1e-15)
    assert tr.gap(1, 0, 0, 0) == 0.0
    assert tr.gap(1, 0, 1, 0) == pytest.approx(abs(tr.dplus[0, 0]))


def test_first_divergence_localises_a_planted_change():
    """first_divergence finds the first round and coordinate at which another
    run's codes leave the oracle's and reports the oracle's gap between the
    two outcomes there: a copy of the oracle's own run has none; a run that
    flips one decision of round 2 is found at that decision with the gap
    |dplus| (or |dminus|, or their difference); a changed initial code is
    found at round 0 with that coordinate's boundary distance; a jump of two
    code steps has an infinite gap."""
    rng = np.random.default_rng(77)
    o = rng.standard_normal(64) * np.linspace(2.0, 0.5, 64)
    B, R = 4, 6
    tr = O.caq_trace(o, B, R)
    assert O.first_divergence(o, B, R, tr.codes_after) == (-1, -1, 0.0)
    for i in (3, 17, 40):
        alt = tr.codes_after.astype(int).copy()
        prev = alt[1, i]
        a = alt[2, i] - prev
        b = 0 if a != 0 else (1 if prev < 2 ** B - 1 else -1)
        alt[2:, i] = prev + b            # the other run decides differently here
        alt[2:, i + 1:] += 0             # later coordinates unchanged
        r, j, m = O.first_divergence(o, B, R, alt)
        assert (r, j) == (2, i)
        d = {0: 0.0, 1: tr.dplus[1, i], -1: tr.dminus[1, i]}
        assert m == pytest.approx(abs(d[a] - d[b]), rel=1e-15)
    alt = tr.codes_after.astype(int).copy()
    alt[:, 9] = np.clip(alt[:, 9] + 1, 0, 2 ** B - 1) if alt[0, 9] < 2 ** B - 1 else alt[:, 9] - 1
    r, j, m = O.first_divergence(o, B, R, alt)
    assert (r, j) == (0, 9) and m == pytest.approx(tr.init_margin[9])
    alt = tr.codes_after.astype(int).copy()
    k = int(np.argmax((alt[0] >= 2) & (alt[0] <= 2 ** B - 3)))
    alt[1:, k] = alt[0, k] + 2
    assert O.first_divergence(o, B, R, alt)[2] == math.inf


# ---------------------------------------------------- multi-stage estimation
def test_segment_sigma_is_the_variance_of_the_segment_inner_product():
    """Sec. 4.3: sigma_Seg^2 = sum_{i in Seg} q[i]^2 sigma_i^2 is the
    variance, over the data vectors, of <o_seg, q_seg>.  Computed here the
    other way round: the empirical (1/N) variance over the fitted rows of
    <W_s (x - c), W_s (q - c)>, through the rotated matrix W and the data."""
    X, _, _ = _power_law(5000, 128, 0.8, seed=21)
    m = O.fit(X, 3.0)
    rng = np.random.default_rng(22)
    Qm = X[rng.choice(5000, 30, replace=False)] + 0.1 * rng.standard_normal((30, 128))
    sig = O.segment_sigma(m, Qm)
    Oproj, _ = O.project(X, m)
    Qr, _ = O.project(Qm, m)
    for j, (off, l, b) in enumerate(m.kept):
        ip = Oproj[:, off:off + l] @ Qr[:, off:off + l].T          # (N, nq)
        var = ip.var(axis=0)                                        # 1/N, as the PCA
        assert np.allclose(sig[:, j] ** 2, var, rtol=1e-9, atol=1e-12)


def test_chebyshev_bound_holds_per_segment():
    """Sec. 4.3: |<o_seg, q_seg>| >= m sigma_Seg with probability <= 1/m^2
    (Chebyshev, the inner product has mean 0 over centred data).  On the
    fitted rows the empirical frequency obeys the bound for every segment
    and every m; for near-normal values it is far below it."""
    X, _, _ = _power_law(6000, 96, 1.0, seed=23)
    m = O.fit(X, 2.0)
    Qm = X[:40]
    sig = O.segment_sigma(m, Qm)
    Oproj, _ = O.project(X, m)
    Qr, _ = O.project(Qm, m)
    for j, (off, l, b) in enumerate(m.kept):
        ip = np.abs(Oproj[:, off:off + l] @ Qr[:, off:off + l].T)
        for mc in (1.5, 2.0, 3.0):
            freq = np.mean(ip >= mc * sig[None, :, j])
            assert freq <= 1.0 / mc ** 2
        assert np.mean(ip >= 2.0 * sig[None, :, j]) < 0.1


def test_staged_estimate_ends_at_the_estimate_and_starts_at_the_prior_bound():
    """Sec. 4.3 multi-stage estimator: after all kept segments it is the
    Sec. 3.2 estimate; before any, |x - c|^2 + |q - c|^2 - 2 m sum_s
    sigma_s(q); each stage swaps one Chebyshev bound for one estimate, so
    the step t -> t+1 is 2 (m sigma_t - est_t), and m = 0 keeps only the
    estimated stages."""
    X, _, _ = _power_law(3000, 128, 0.8, seed=24)
    m = O.fit(X, 4.0)
    e = O.encode(X[:50], m, rounds=6)
    Qm = X[-20:]
    k = len(m.kept)
    st = O.estimate_staged(m, e.codes, e.factors, Qm, 2.0)
    assert st.shape == (20, 50, k + 1)
    full = O.estimate(m, e.codes, e.factors, Qm)
    assert np.allclose(st[:, :, k], full, rtol=1e-12, atol=1e-9)
    Qc = Qm - m.mean
    base = e.factors[None, :, 0] + np.sum(Qc * Qc, axis=1)[:, None]
    sig = O.segment_sigma(m, Qm)
    assert np.allclose(st[:, :, 0], base - 4.0 * sig.sum(axis=1)[:, None], rtol=1e-12)
    est = O.segment_estimates(m, e.codes, e.factors, Qm)
    for t in range(k):
        step = st[:, :, t + 1] - st[:, :, t]
        assert np.allclose(step, 2.0 * (2.0 * sig[:, t][:, None] - est[:, :, t]), rtol=1e-9,
                           atol=1e-9)
    # the stage-t bound is a lower bound of the exact distance for most pairs
    ex = O.exact_dist(X[:50], Qm)
    assert np.mean(st[:, :, 0] <= ex) >= 0.75
    st0 = O.estimate_staged(m, e.codes, e.factors, Qm, 0.0)
    assert np.allclose(st0[:, :, 0], base, rtol=1e-12)
