"""Element-by-element comparison of the library's codes and factors with the
FP64 oracle's, shared by the GPU parity tests.

Bars (FP32 path):
  * >= 99.9% of codes identical;
  * every vector-segment whose codes differ is traced to the FIRST decision
    at which the library's run leaves the oracle's (the first round r whose
    codes differ, then the first coordinate in it; r = 0 is the initial
    code), and the oracle's own margin at that decision must be < 1e-5:
    cosine units |L(c + a) - L(c + b)| between the two outcomes for an
    adjustment trial (Sec. 3.1 Algorithm 1), and the distance to the nearest
    interval boundary over |o_s| for an initial code (Eq. find_nearest_code).
    The library's codes after r rounds come from re-running it with r rounds
    (a round without a move ends a segment early, which changes nothing);
  * per-vector relative quantization error within 1e-4 of the oracle's, on
    every vector;
  * |o_s| within 1e-5 relative; cos_s within 1e-5 where the codes agree;
  * mean relative distance-estimate error within 1e-4 of the oracle's.
"""
import numpy as np

import oracle as O

CODE_AGREE = 0.999
MARGIN = 1e-5
EPS_TOL = 1e-4
DIST_TOL = 1e-4


def gpu_codes_by_round(model, mo, run, rounds):
    """The library's unpacked codes after r = 0 .. rounds rounds: `run()`
    encodes the rows with the model's current round count and returns the
    packed codes; the model's round count is restored afterwards."""
    out = []
    try:
        for r in range(rounds + 1):
            model.set_rounds(r)
            out.append(O.unpack(np.ascontiguousarray(run()), mo))
    finally:
        model.set_rounds(rounds)
    return out


def localise_mismatches(mo, O_rows, mism, after, rounds):
    """For each mismatching (row, kept segment) the oracle's margin at the
    first divergent decision (see the module docstring): an array of
    (row, segment, round, coordinate, margin)."""
    rows = []
    for v, j in zip(*np.nonzero(mism)):
        off, l, b = mo.kept[j]
        o = O_rows[v, off:off + l]
        other = [a[v, off:off + l] for a in after]
        r, i, m = O.first_divergence(o, b, rounds, other)
        rows.append((v, j, r, i, m))
    return rows


def check_codes(mo, eo, codes_gpu, factors_gpu, O_rows=None, after=None, rounds=6,
                agree_min=CODE_AGREE, margin=MARGIN, label=""):
    """Codes and factors of the library against the oracle's (module
    docstring).  O_rows: the rows' projection the oracle encoded (FP64,
    n x d_kept); after: the library's codes after 0 .. rounds rounds
    (gpu_codes_by_round), or a callable that returns them, called only when
    some codes differ.  Returns a dict of the agreement statistics, which
    it also prints."""
    codes = O.unpack(codes_gpu, mo)
    # padding bits of the packed planes are zero: pack(unpack(x)) == x
    assert np.array_equal(O.pack(codes, mo), codes_gpu)
    eq = codes == eo.codes
    frac = float(eq.mean()) if eq.size else 1.0
    assert frac >= agree_min, "%s code agreement %.6f" % (label, frac)
    k = len(mo.kept)
    mism = np.zeros((codes.shape[0], k), dtype=bool)
    for j, (off, l, b) in enumerate(mo.kept):
        mism[:, j] = ~eq[:, off:off + l].all(axis=1)
    worst = 0.0
    per_round = {}
    if mism.any():
        assert O_rows is not None and after is not None, "mismatches need the per-round codes"
        if callable(after):
            after = after()
        # the re-run with `rounds` rounds is the encode under test
        assert np.array_equal(after[rounds], codes), "re-run codes differ from the encode's"
        loc = localise_mismatches(mo, O_rows, mism, after, rounds)
        for v, j, r, i, m in loc:
            assert r >= 0, "row %d segment %d differs but no round diverges" % (v, j)
            per_round[r] = per_round.get(r, 0) + 1
        worst = max(m for *_, m in loc)
        bad = [x for x in loc if not x[4] < margin]
        assert not bad, "%s divergence at oracle margin >= %g: %s" % (label, margin, bad[:5])
    f = factors_gpu.astype(np.float64)
    ref = eo.factors
    nr_g, nr_o = f[:, 1::2], ref[:, 1::2]
    assert np.allclose(nr_g, nr_o, rtol=1e-5, atol=1e-6 * max(1.0, nr_o.max()))
    assert np.allclose(f[:, 0], ref[:, 0], rtol=1e-5, atol=1e-6 * max(1.0, ref[:, 0].max()))
    cg, co = f[:, 2::2], ref[:, 2::2]
    assert np.all((np.abs(cg - co) <= 1e-5) | mism), "cos factor off where codes agree"
    if mism.any():
        # past a near-tie both runs are valid CAQ results: the library's
        # cosine is at least its initial code's (to the 1e-5 rounding of an
        # FP32 cosine factor) and close to the oracle's
        assert np.all(cg[mism] >= eo.init_cos[mism] - 1e-5)
        assert np.all(np.abs(cg[mism] - co[mism]) <= 1e-3)
    eg, eo_ = O.quant_error(f, mo), O.quant_error(ref, mo)
    de = np.abs(eg - eo_)
    rowm = mism.any(axis=1)
    stats = {
        "label": label, "codes": int(eq.size), "codes_differ": int((~eq).sum()),
        "agreement": frac, "vector_segments": int(mism.size),
        "vector_segments_differ": int(mism.sum()), "divergence_rounds": per_round,
        "worst_divergence_margin": float(worst),
        "max_eps_diff": float(de.max(initial=0.0)),
        "max_eps_diff_where_codes_differ": float(de[rowm].max(initial=0.0)),
        "mean_eps_diff": float(abs(eg.mean() - eo_.mean())),
    }
    print("PARITY %s" % stats)
    assert de.max(initial=0.0) <= EPS_TOL, "%s per-vector eps diff %.3g" % (label, de.max())
    assert abs(eg.mean() - eo_.mean()) <= EPS_TOL
    return stats
