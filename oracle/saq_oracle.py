"""Plain FP64 CPU oracle of SAQ -- TEST INFRASTRUCTURE ONLY.

This module restates, step by step and in FP64, what SAQ computes
(arXiv 2509.12086).  It exists to check the CUDA library; only tests/, the
smoke check and the CPU-baseline leg of bench.py may import it.  It shares no
code with the library, and it never takes an input or an expected value from
the library.

Paper passages followed (section / equation / algorithm):
  * Sec. 2.2 Eq. 2-3    distance from norms and an inner product about c
  * Sec. 3.1 Eq. rotate o = P (o_r - c)
  * Sec. 3.1 Eq. find_nearest_code, Eq. adj-obj, Algorithm 1 (CAQ)
  * Sec. 3.2 Eq. estimator_inner_product and the estimator
              <o,q> ~ <o_bar_a,q> / <o_bar_a,o> * |o|^2
  * Sec. 4.1 PCA fit, sigma_1 >= ... >= sigma_D, segment rotations
  * Sec. 4.2 Eq. seg-err (empirical-variance form, no pi), Algorithm 2,
              segments in multiples of 64, fewest segments within 0.1%
  * Sec. 5.1 one combined PCA + rotation matrix

Readings where the paper is silent or ambiguous are listed where they are
used; the same list is kept with the design notes of the repository.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

from . import build as _build

_lib = None


def _c():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.saq_oracle_caq_segment.argtypes = [
            dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p, dp, dp, ip, dp,
            dp, dp]
        lib.saq_oracle_caq_segment.restype = ctypes.c_int
        lib.saq_oracle_encode.argtypes = [
            dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ip, ip, ip,
            ctypes.c_int, ctypes.c_int, u8p, dp, dp, ip, dp, dp, dp]
        lib.saq_oracle_encode.restype = None
        lib.saq_oracle_plan.argtypes = [
            dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
            ctypes.c_double, ip, ip, ip, ip, dp, dp, i64p]
        lib.saq_oracle_plan.restype = ctypes.c_int
        lib.saq_oracle_max_threads.restype = ctypes.c_int
        lib.saq_oracle_caq_trace.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             u8p, dp, dp, dp]
        lib.saq_oracle_caq_trace.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def max_threads() -> int:
    return int(_c().saq_oracle_max_threads())


# --------------------------------------------------------------------------
# Fit: PCA (Sec. 4.1)
# --------------------------------------------------------------------------
def pca(X: np.ndarray, chunk: int = 65536) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Mean c, eigenvalues sigma^2 (descending) and eigenvectors (columns) of
    the covariance (1/N) sum (x - c)(x - c)^T, all FP64 (Sec. 4.1: learn a PCA
    rotation so that sigma_1 >= sigma_2 >= ... >= sigma_D).

    Readings: the covariance uses 1/N (the plan is scale invariant); equal
    eigenvalues keep the solver's order (stable sort); each eigenvector is
    signed so that its largest-magnitude component (lowest index on ties) is
    positive.
    """
    n, d = X.shape
    c = np.zeros(d)
    for i in range(0, n, chunk):
        c += X[i:i + chunk].astype(np.float64).sum(axis=0)
    c /= n
    C = np.zeros((d, d))
    for i in range(0, n, chunk):
        Y = X[i:i + chunk].astype(np.float64) - c
        C += Y.T @ Y
    C /= n
    w, V = np.linalg.eigh(C)
    order = np.argsort(-w, kind="stable")
    w = w[order]
    V = V[:, order]
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(d)])
    sgn[sgn == 0] = 1.0
    V = V * sgn
    return c, np.maximum(w, 0.0), V


# --------------------------------------------------------------------------
# Fit: quantization plan (Sec. 4.2, Algorithm 2)
# --------------------------------------------------------------------------
@dataclass
class Plan:
    segments: List[Tuple[int, int, int]]  # (start, len, bits), cover [0, D)
    error: float                           # ERROR(P), Eq. seg-err summed
    min_error: float                       # least error over all plans
    cost: int                              # C(P) = sum B |Seg|


def plan_dp(sig2: np.ndarray, quota_bits: int, g: int = 64, max_bits: int = 8,
            tie_frac: float = 1e-3) -> Plan:
    """Algorithm 2 with ERROR(Seg, B) = sum sigma_i^2 * 2^-B.

    Readings: the cost update uses the segment length (B * |Seg|, consistent
    with C(P)); segments are non-empty multiples of g except a final
    remainder; valid bits are 0..max_bits with B = 0 dropping the segment and
    costing its full variance; the plan chosen has the fewest segments among
    plans within (1 + tie_frac) of the least error, then the least error,
    then the least cost, then the first found in enumeration order.
    """
    sig2 = np.ascontiguousarray(sig2, dtype=np.float64)
    D = sig2.shape[0]
    ng = (D + g - 1) // g
    st = np.zeros(ng, dtype=np.int32)
    ln = np.zeros(ng, dtype=np.int32)
    bt = np.zeros(ng, dtype=np.int32)
    ns = ctypes.c_int()
    err = ctypes.c_double()
    emin = ctypes.c_double()
    cost = ctypes.c_int64()
    rc = _c().saq_oracle_plan(_ptr(sig2, ctypes.c_double), D, g,
                              int(quota_bits), max_bits, tie_frac,
                              _ptr(st, ctypes.c_int), _ptr(ln, ctypes.c_int),
                              _ptr(bt, ctypes.c_int), ctypes.byref(ns),
                              ctypes.byref(err), ctypes.byref(emin),
                              ctypes.byref(cost))
    if rc != 0:
        raise ValueError("plan search failed")
    k = ns.value
    segs = [(int(st[i]), int(ln[i]), int(bt[i])) for i in range(k)]
    return Plan(segs, err.value, emin.value, int(cost.value))


def plan_error(sig2: np.ndarray, segments) -> float:
    """ERROR(P) of an explicit plan (Eq. seg-err summed over segments)."""
    return float(sum(np.sum(sig2[s:s + l]) * 2.0 ** (-b) for s, l, b in segments))


# --------------------------------------------------------------------------
# Fit: segment rotations and the combined matrix (Sec. 4.1, Sec. 5.1)
# --------------------------------------------------------------------------
def haar(n: int, rng: np.random.Generator) -> np.ndarray:
    """Random orthonormal matrix (Sec. 2.2 / Sec. 4.1): QR of a Gaussian
    matrix with the columns of Q signed by diag(R), which makes it Haar
    distributed (reading: 'random orthonormal' is Haar)."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


@dataclass
class Model:
    d: int
    mean: np.ndarray                      # c, (d,)
    W: np.ndarray                         # (d_kept, d): rows of blockdiag(R_s) V_s^T
    plan: List[Tuple[int, int, int]]      # all segments, PCA dimension order
    sig2: np.ndarray = None               # (d,) PCA eigenvalues
    kept: List[Tuple[int, int, int]] = field(default_factory=list)  # (off, len, bits)
    V: np.ndarray = None                  # (d, d) PCA eigenvectors (columns), if known

    def __post_init__(self):
        if not self.kept:
            off = 0
            for s, l, b in self.plan:
                if b > 0:
                    self.kept.append((off, l, b))
                    off += l

    @property
    def d_kept(self) -> int:
        return int(sum(l for _, l, _ in self.kept))

    @property
    def code_bytes(self) -> int:
        return int(sum(b * ((l + 63) // 64) * 8 for _, l, b in self.kept))

    @property
    def factor_count(self) -> int:
        return 1 + 2 * len(self.kept)


def build_matrix(V: np.ndarray, plan, seed: int) -> np.ndarray:
    """W = blockdiag(R_s) V_kept^T: the PCA projection followed by one random
    rotation per kept segment, combined into one matrix (Sec. 5.1).  Segments
    with B = 0 are discarded (Sec. 4.2: B = 0 keeps nothing)."""
    rng = np.random.default_rng(seed)
    rows = []
    for s, l, b in plan:
        if b == 0:
            continue
        R = haar(l, rng)
        rows.append(R @ V[:, s:s + l].T)
    d = V.shape[0]
    return np.concatenate(rows, axis=0) if rows else np.zeros((0, d))


def fit(X: np.ndarray, avg_bits: float, g: int = 64, max_bits: int = 8,
        tie_frac: float = 1e-3, seed: int = 4) -> Model:
    """Whole fit: PCA, plan with Q_quota = round(avg_bits * D) (reading for
    fractional averages), rotations, combined matrix."""
    c, sig2, V = pca(X)
    d = X.shape[1]
    plan = plan_dp(sig2, int(round(avg_bits * d)), g, max_bits, tie_frac)
    W = build_matrix(V, plan.segments, seed)
    return Model(d=d, mean=c, W=W, plan=plan.segments, sig2=sig2, V=V)


# --------------------------------------------------------------------------
# Encode (Sec. 3.1, Algorithm 1; Sec. 4.2 last paragraph)
# --------------------------------------------------------------------------
def project(X: np.ndarray, model: Model) -> Tuple[np.ndarray, np.ndarray]:
    """o = W (x - c) for the kept dimensions, and |x - c|^2 over all d."""
    Y = X.astype(np.float64) - model.mean
    return Y @ model.W.T, np.einsum("ij,ij->i", Y, Y)


@dataclass
class Encoded:
    codes: np.ndarray          # (n, d_kept) uint8, one code per kept coordinate
    factors: np.ndarray        # (n, 1 + 2k): |x-c|^2, then (|o_s|, cos_s)
    accepts: np.ndarray        # (n, k, rounds) accepted moves per round
    min_trial_margin: np.ndarray   # (n, k)
    min_init_margin: np.ndarray    # (n, k)
    init_cos: np.ndarray           # (n, k)

    @property
    def min_margin(self) -> np.ndarray:
        return np.minimum(self.min_trial_margin, self.min_init_margin)


def caq_segment(o: np.ndarray, B: int, rounds: int):
    """CAQ of one segment; returns (codes, norm, cos, accepts, min trial
    margin, min init margin, init cos)."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    n = o.shape[0]
    code = np.zeros(n, dtype=np.uint8)
    acc = np.zeros(max(rounds, 1), dtype=np.int32)
    nrm, cs, mt, mi, ic = (ctypes.c_double() for _ in range(5))
    _c().saq_oracle_caq_segment(_ptr(o, ctypes.c_double), n, B, rounds,
                                _ptr(code, ctypes.c_uint8), ctypes.byref(nrm),
                                ctypes.byref(cs), _ptr(acc, ctypes.c_int),
                                ctypes.byref(mt), ctypes.byref(mi),
                                ctypes.byref(ic))
    return code, nrm.value, cs.value, acc[:rounds].copy(), mt.value, mi.value, ic.value


@dataclass
class Trace:
    """Every decision of one run of Algorithm 1 on one segment."""
    codes_after: np.ndarray   # (rounds + 1, len) uint8: initial codes, then after each round
    init_margin: np.ndarray   # (len,) distance of o_i to its nearest interior boundary / |o|
    dplus: np.ndarray         # (rounds, len) L(x + Delta e_i) - L(x) when round r reaches i
    dminus: np.ndarray        # (rounds, len) L(x - Delta e_i) - L(x) from the same state

    def gap(self, r: int, i: int, a: int, b: int) -> float:
        """|L(c + a) - L(c + b)| for moves a, b in {-1, 0, +1} of coordinate i
        from the state at which round r (1-based) reaches it: how far apart
        in the objective two outcomes of that decision are (inf if a move
        leaves the code range)."""
        d = {0: 0.0, 1: self.dplus[r - 1, i], -1: self.dminus[r - 1, i]}
        if not (np.isfinite(d[a]) and np.isfinite(d[b])):
            return math.inf
        return abs(d[a] - d[b])


def caq_trace(o: np.ndarray, B: int, rounds: int) -> Trace:
    """Replay CAQ on one segment (Sec. 3.1, Algorithm 1) and record every
    decision: the codes after each round and, for each (round, coordinate),
    the objective change of either move from the state the scan is in when
    it reaches that coordinate.  The run itself is the one caq_segment
    performs; the record only observes it."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    n = o.shape[0]
    ca = np.zeros((rounds + 1, n), dtype=np.uint8)
    im = np.zeros(n)
    dp_ = np.zeros((max(rounds, 1), n))
    dm = np.zeros((max(rounds, 1), n))
    _c().saq_oracle_caq_trace(_ptr(o, ctypes.c_double), n, B, rounds,
                              _ptr(ca, ctypes.c_uint8), _ptr(im, ctypes.c_double),
                              _ptr(dp_, ctypes.c_double), _ptr(dm, ctypes.c_double))
    return Trace(ca, im, dp_[:rounds], dm[:rounds])


def first_divergence(o: np.ndarray, B: int, rounds: int, other_after) -> Tuple[int, int, float]:
    """Where another run of Algorithm 1 on segment o first leaves the
    oracle's, and how close that decision was.

    other_after[r] holds the other run's codes of this segment after r rounds
    (r = 0: initial codes).  Returns (r, i, margin) for the first round r and,
    within it, the first coordinate i whose code differs.  Up to that point
    both runs made the same decisions, so both arrive at coordinate i in the
    same state, and the margin is the oracle's objective gap between the two
    outcomes there: for r = 0 the distance of o_i to the nearest interval
    boundary of the initial grid over |o|; for r >= 1, |L(c + a) - L(c + b)|
    for the oracle's move a and the other run's move b (inf if b is not a
    single step inside the code range).  (-1, -1, 0.0) if the runs agree."""
    tr = caq_trace(o, B, rounds)
    for r in range(rounds + 1):
        mine = tr.codes_after[r]
        theirs = np.asarray(other_after[r]).astype(np.int64)
        diff = np.nonzero(mine.astype(np.int64) != theirs)[0]
        if diff.size == 0:
            continue
        i = int(diff[0])
        if r == 0:
            return 0, i, float(tr.init_margin[i])
        prev = int(tr.codes_after[r - 1, i])
        a = int(mine[i]) - prev
        b = int(theirs[i]) - prev
        if b not in (-1, 0, 1):
            return r, i, math.inf
        return r, i, float(tr.gap(r, i, a, b))
    return -1, -1, 0.0


def encode_projected(O: np.ndarray, norms2: np.ndarray, model: Model,
                     rounds: int, nthreads: int = 0) -> Encoded:
    """Quantize each kept segment of each projected vector separately with
    CAQ (Sec. 4.2 last paragraph) and collect the stored factors."""
    O = np.ascontiguousarray(O, dtype=np.float64)
    n, dk = O.shape
    k = len(model.kept)
    off = np.array([s[0] for s in model.kept], dtype=np.int32)
    ln = np.array([s[1] for s in model.kept], dtype=np.int32)
    bt = np.array([s[2] for s in model.kept], dtype=np.int32)
    codes = np.zeros((n, dk), dtype=np.uint8)
    norms = np.zeros((n, k))
    coss = np.zeros((n, k))
    r = max(rounds, 1)
    acc = np.zeros((n, k, r), dtype=np.int32)
    mt = np.zeros((n, k))
    mi = np.zeros((n, k))
    ic = np.zeros((n, k))
    if n and k:
        _c().saq_oracle_encode(_ptr(O, ctypes.c_double), n, dk, k,
                               _ptr(off, ctypes.c_int), _ptr(ln, ctypes.c_int),
                               _ptr(bt, ctypes.c_int), rounds, nthreads,
                               _ptr(codes, ctypes.c_uint8),
                               _ptr(norms, ctypes.c_double),
                               _ptr(coss, ctypes.c_double),
                               _ptr(acc, ctypes.c_int), _ptr(mt, ctypes.c_double),
                               _ptr(mi, ctypes.c_double), _ptr(ic, ctypes.c_double))
    factors = np.zeros((n, 1 + 2 * k))
    factors[:, 0] = norms2
    factors[:, 1::2] = norms
    factors[:, 2::2] = coss
    return Encoded(codes, factors, acc[:, :, :rounds], mt, mi, ic)


def encode(X: np.ndarray, model: Model, rounds: int = 6,
           nthreads: int = 0) -> Encoded:
    O, n2 = project(X, model)
    return encode_projected(O, n2, model, rounds, nthreads)


# --------------------------------------------------------------------------
# Storage layout of the codes (reading: the paper leaves the bit layout open)
# --------------------------------------------------------------------------
def pack(codes: np.ndarray, model: Model) -> np.ndarray:
    """Per vector, per kept segment in plan order, B bit-planes, most
    significant first; plane p holds bit (B-1-p) of every code of the segment
    as ceil(len/64) little-endian 64-bit words (coordinate i -> word i // 64,
    bit i % 64).  Taking the first b planes of a segment gives the b-bit
    prefix code floor(c / 2^(B-b)) of Sec. 3.2."""
    n = codes.shape[0]
    out = []
    for off, l, b in model.kept:
        words = (l + 63) // 64
        seg = codes[:, off:off + l]
        for p in range(b):
            bits = ((seg >> (b - 1 - p)) & 1).astype(np.uint8)
            pad = np.zeros((n, words * 64), dtype=np.uint8)
            pad[:, :l] = bits
            out.append(np.packbits(pad, axis=1, bitorder="little"))
    if not out:
        return np.zeros((n, 0), dtype=np.uint8)
    return np.ascontiguousarray(np.concatenate(out, axis=1))


def unpack(packed: np.ndarray, model: Model) -> np.ndarray:
    n = packed.shape[0]
    codes = np.zeros((n, model.d_kept), dtype=np.uint8)
    pos = 0
    for off, l, b in model.kept:
        words = (l + 63) // 64
        for p in range(b):
            plane = packed[:, pos:pos + words * 8]
            bits = np.unpackbits(plane, axis=1, bitorder="little")[:, :l]
            codes[:, off:off + l] |= (bits << (b - 1 - p)).astype(np.uint8)
            pos += words * 8
    return codes


# --------------------------------------------------------------------------
# Distance estimation (Sec. 2.2 Eq. 3, Sec. 3.2)
# --------------------------------------------------------------------------
def estimate(model: Model, codes: np.ndarray, factors: np.ndarray,
             Q: np.ndarray, prefix_bits: int = 0) -> np.ndarray:
    """Estimated squared distances (nq, n).

    Per kept segment s, with u = 2c - (2^B - 1) (the quantized vector o_bar_a
    up to the positive factor Delta / 2, Sec. 3.1):
        <o_s, q_s>  ~  |o_s| <u, q_s> / (|u| cos_s)
    which is the estimator <o_bar_a, q> / <o_bar_a, o> * |o|^2 of Sec. 3.2
    written with the stored factors |o_s| and cos_s = <o_bar_a, o>/(|o_bar_a||o|).
    Then Eq. 3: |o_r - q_r|^2 = |o_r - c|^2 + |q_r - c|^2 - 2 <o_r - c, q_r - c>,
    with dropped segments contributing nothing to the inner product.

    prefix_bits > 0 uses the b-bit prefix floor(c / 2^(B-b)) of each segment
    with b = min(prefix_bits, B) (progressive approximation, Sec. 3.2); the
    grid offset changes to 2^b - 1 and the stored factors are reused.
    """
    Qc = Q.astype(np.float64) - model.mean
    qr = Qc @ model.W.T
    qn2 = np.einsum("ij,ij->i", Qc, Qc)
    est = np.zeros((Q.shape[0], codes.shape[0]))
    for j, (off, l, b) in enumerate(model.kept):
        c = codes[:, off:off + l].astype(np.float64)
        bb = b
        if prefix_bits > 0 and prefix_bits < b:
            bb = prefix_bits
            c = np.floor(c / 2.0 ** (b - bb))
        u = 2.0 * c - (2.0 ** bb - 1.0)
        un = np.sqrt(np.sum(u * u, axis=1))
        nrm = factors[:, 1 + 2 * j]
        cs = factors[:, 2 + 2 * j]
        scale = np.where(nrm > 0, nrm / (un * np.where(cs != 0, cs, 1.0)), 0.0)
        est += (qr[:, off:off + l] @ u.T) * scale[None, :]
    return factors[None, :, 0] + qn2[:, None] - 2.0 * est


# --------------------------------------------------------------------------
# Multi-stage estimation (Sec. 4.3)
# --------------------------------------------------------------------------
def kept_basis(model: Model) -> np.ndarray:
    """(d_kept, d): the PCA directions v_i^T of the kept dimensions, plan
    order (the rows W_s mixes with the segment rotation R_s)."""
    rows = [model.V[:, s:s + l].T for s, l, b in model.plan if b > 0]
    return np.concatenate(rows, axis=0) if rows else np.zeros((0, model.d))


def segment_sigma(model: Model, Q: np.ndarray) -> np.ndarray:
    """(nq, k): sigma_Seg(q) of every kept segment, Sec. 4.3:
        sigma_Seg^2 = sum_{i in Seg} q[i]^2 sigma_i^2
    with q in the PCA coordinates, q[i] = v_i^T (q_r - c), and sigma_i^2 the
    variance of PCA dimension i over the dataset.  It is the variance of
    <o_seg, q_seg> over the data vectors (the segment rotation R_s does not
    change an inner product)."""
    Qp = (Q.astype(np.float64) - model.mean) @ model.V      # (nq, d) PCA coordinates
    out = np.zeros((Q.shape[0], len(model.kept)))
    j = 0
    for s, l, b in model.plan:
        if b == 0:
            continue
        out[:, j] = np.sqrt(np.sum(Qp[:, s:s + l] ** 2 * model.sig2[None, s:s + l], axis=1))
        j += 1
    return out


def segment_estimates(model: Model, codes: np.ndarray, factors: np.ndarray,
                      Q: np.ndarray) -> np.ndarray:
    """(nq, n, k): est_s = |o_s| <u_s, q_s> / (|u_s| cos_s) per kept segment
    (the per-segment term of the Sec. 3.2 estimator)."""
    qr = (Q.astype(np.float64) - model.mean) @ model.W.T
    out = np.zeros((Q.shape[0], codes.shape[0], len(model.kept)))
    for j, (off, l, b) in enumerate(model.kept):
        u = 2.0 * codes[:, off:off + l].astype(np.float64) - (2.0 ** b - 1.0)
        un = np.sqrt(np.sum(u * u, axis=1))
        nrm = factors[:, 1 + 2 * j]
        cs = factors[:, 2 + 2 * j]
        scale = np.where(nrm > 0, nrm / (un * np.where(cs != 0, cs, 1.0)), 0.0)
        out[:, :, j] = (qr[:, off:off + l] @ u.T) * scale[None, :]
    return out


def estimate_staged(model: Model, codes: np.ndarray, factors: np.ndarray,
                    Q: np.ndarray, m_conf: float) -> np.ndarray:
    """(nq, n, k + 1) multi-stage lower bounds of the squared distance,
    Sec. 4.3: stages take the kept segments in plan order (decreasing
    variance).  After t stages the first t segments contribute their
    estimates and each remaining one its Chebyshev bound m * sigma_Seg(q)
    (|<o_seg, q_seg>| < m sigma_Seg with probability >= 1 - 1/m^2):
        lb_t = |o_r - c|^2 + |q_r - c|^2
               - 2 (sum_{s < t} est_s + m sum_{s >= t} sigma_s(q)).
    lb_k is the estimate of Sec. 3.2; dropped segments contribute nothing,
    as in that estimate."""
    est = segment_estimates(model, codes, factors, Q)
    sig = segment_sigma(model, Q)
    Qc = Q.astype(np.float64) - model.mean
    base = factors[None, :, 0] + np.einsum("ij,ij->i", Qc, Qc)[:, None]
    k = len(model.kept)
    out = np.zeros((Q.shape[0], codes.shape[0], k + 1))
    for t in range(k + 1):
        done = est[:, :, :t].sum(axis=2)
        rest = m_conf * sig[:, t:].sum(axis=1)
        out[:, :, t] = base - 2.0 * (done + rest[:, None])
    return out


def exact_dist(X: np.ndarray, Q: np.ndarray) -> np.ndarray:
    X = X.astype(np.float64)
    Q = Q.astype(np.float64)
    return (np.einsum("ij,ij->i", Q, Q)[:, None] + np.einsum("ij,ij->i", X, X)[None, :]
            - 2.0 * Q @ X.T)


def relative_error(est: np.ndarray, exact: np.ndarray) -> np.ndarray:
    """|d2_est - d2| / d2 (Sec. 5, performance metrics)."""
    return np.abs(est - exact) / np.maximum(exact, 1e-300)


def quant_error(factors: np.ndarray, model: Model) -> np.ndarray:
    """Per-vector relative quantization error
        [sum_kept |o_s|^2 (1 - cos_s^2) + sum_dropped |o_s|^2] / |x - c|^2,
    the squared residual of the best rescaling of o_bar_a along its direction
    for each kept segment plus the energy of the dropped dimensions."""
    n2 = factors[:, 0]
    nr = factors[:, 1::2]
    cs = factors[:, 2::2]
    kept = np.sum(nr * nr, axis=1)
    res = np.sum(nr * nr * (1.0 - cs * cs), axis=1) + np.maximum(n2 - kept, 0.0)
    return np.where(n2 > 0, res / np.where(n2 > 0, n2, 1.0), 0.0)
