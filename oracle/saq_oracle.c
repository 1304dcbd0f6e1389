/*
 * saq_oracle.c -- plain FP64 CPU oracle for SAQ (Segmented CAQ).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant generator with
 * the CUDA library.
 *
 * It holds the two parts of the oracle that need per-element loops:
 *   - code adjustment of one vector segment (Sec. 3.1, Eq. find_nearest_code,
 *     Eq. adj-obj, Algorithm 1), with decision margins logged;
 *   - the quantization-plan dynamic program (Sec. 4.2, Eq. seg-err,
 *     Algorithm 2) extended by a segment-count index for the "fewest segments
 *     within 0.1% of the minimum" rule stated after Algorithm 2.
 * Everything is FP64, single-threaded per vector; only the outer loop over
 * vectors runs in parallel (OpenMP), which changes no result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Cosine objective of Eq. adj-obj, L(x, o) = <x,o> / (|x| |o|), evaluated from
 * the running dot product and squared norm of x (the O(1) incremental update
 * described after Algorithm 1). */
static double objective(double dot, double sq, double norm_o) {
    return dot / (sqrt(sq) * norm_o);
}

/*
 * Algorithm 1 on one segment, shared by the plain entry point below and by
 * the replay that records every decision (saq_oracle_caq_trace).  The trace
 * outputs may be NULL; they only observe the run and change nothing in it:
 *   codes_after[(r + 1) * len + i]  code of coordinate i after round r
 *                                   (row 0: the initial code)
 *   init_margin[i]                  distance of o[i] to the nearest interior
 *                                   interval boundary of the initial grid,
 *                                   divided by |o| (as *min_init_margin)
 *   dplus[r * len + i], dminus[r * len + i]
 *                                   L(x + Delta e_i) - L(x) and
 *                                   L(x - Delta e_i) - L(x) evaluated at the
 *                                   state x reached when round r arrives at
 *                                   coordinate i, before its +Delta trial;
 *                                   -INFINITY where the move leaves
 *                                   [-vmax, vmax].  dplus is the algorithm's
 *                                   own +Delta trial; dminus is its -Delta
 *                                   trial whenever +Delta was rejected.
 */
static int caq_run(const double *o, int len, int B, int rounds,
                   uint8_t *code, double *norm_out, double *cos_out,
                   int *accepts, double *min_trial_margin,
                   double *min_init_margin, double *init_cos,
                   uint8_t *codes_after, double *init_margin,
                   double *dplus, double *dminus) {
    int i, r, total = 0;
    const int cmax = (1 << B) - 1;
    double vmax = 0.0, nrm2 = 0.0;
    for (i = 0; i < len; ++i) {
        double a = fabs(o[i]);
        if (a > vmax) vmax = a;
        nrm2 += o[i] * o[i];
    }
    for (r = 0; r < rounds; ++r) accepts[r] = 0;
    *min_trial_margin = INFINITY;
    *min_init_margin = INFINITY;
    if (vmax == 0.0) {
        /* All-zero segment: the paper is silent.  Reading: codes 0, norm 0,
         * cosine 1, and the estimator contributes nothing for it. */
        for (i = 0; i < len; ++i) code[i] = 0;
        *norm_out = 0.0;
        *cos_out = 1.0;
        *init_cos = 1.0;
        if (codes_after)
            memset(codes_after, 0, (size_t)(rounds + 1) * (size_t)len);
        if (init_margin)
            for (i = 0; i < len; ++i) init_margin[i] = INFINITY;
        if (dplus)
            for (i = 0; i < rounds * len; ++i) dplus[i] = dminus[i] = -INFINITY;
        return 0;
    }
    const double norm = sqrt(nrm2);
    /* Eq. find_nearest_code: 2^B intervals of width Delta over [-vmax, vmax]. */
    const double delta = 2.0 * vmax / (double)(1 << B);
    double *x = (double *)malloc(sizeof(double) * (size_t)len);
    int *c = (int *)malloc(sizeof(int) * (size_t)len);
    double dot = 0.0, sq = 0.0;
    for (i = 0; i < len; ++i) {
        double t = (o[i] + vmax) / delta;
        int ci = (int)floor(t);
        /* o[i] == vmax gives 2^B: clamp to the top code (reading of the
         * closed interval end). */
        if (ci > cmax) ci = cmax;
        if (ci < 0) ci = 0;
        c[i] = ci;
        /* distance to the nearest interior boundary k = 1 .. 2^B - 1 */
        double kb = floor(t + 0.5);
        if (kb < 1.0) kb = 1.0;
        if (kb > (double)cmax) kb = (double)cmax;
        if (cmax >= 1) {
            double m = fabs(t - kb) * delta / norm;
            if (m < *min_init_margin) *min_init_margin = m;
            if (init_margin) init_margin[i] = m;
        }
        /* quantized value o_bar[i] = Delta (c + 0.5) - vmax */
        x[i] = delta * ((double)ci + 0.5) - vmax;
        dot += x[i] * o[i];
        sq += x[i] * x[i];
    }
    *init_cos = objective(dot, sq, norm);
    if (codes_after)
        for (i = 0; i < len; ++i) codes_after[i] = (uint8_t)c[i];

    /* Algorithm 1: coordinate-descent rounds.  For each coordinate in order,
     * try +Delta and then -Delta; keep a move iff the new value stays inside
     * [-vmax, vmax] and the cosine strictly increases. */
    for (r = 0; r < rounds; ++r) {
        for (i = 0; i < len; ++i) {
            if (dplus) {
                /* both moves from the state at the start of this step */
                const double l0 = objective(dot, sq, norm);
                for (int s = 0; s < 2; ++s) {
                    const double step = (s == 0) ? delta : -delta;
                    const int cn = c[i] + ((s == 0) ? 1 : -1);
                    double *out = (s == 0) ? dplus : dminus;
                    if (cn < 0 || cn > cmax) {
                        out[(size_t)r * len + i] = -INFINITY;
                        continue;
                    }
                    const double xn = x[i] + step;
                    out[(size_t)r * len + i] =
                        objective(dot + step * o[i], sq - x[i] * x[i] + xn * xn, norm) - l0;
                }
            }
            for (int s = 0; s < 2; ++s) {
                const double step = (s == 0) ? delta : -delta;
                const int cn = c[i] + ((s == 0) ? 1 : -1);
                const double xn = x[i] + step;
                /* x'[i] in [-vmax, vmax]  <=>  0 <= c' <= 2^B - 1 */
                if (cn < 0 || cn > cmax) continue;
                const double dot_n = dot + step * o[i];
                const double sq_n = sq - x[i] * x[i] + xn * xn;
                const double l_old = objective(dot, sq, norm);
                const double l_new = objective(dot_n, sq_n, norm);
                const double m = fabs(l_new - l_old);
                if (m < *min_trial_margin) *min_trial_margin = m;
                if (l_new > l_old) {
                    x[i] = xn;
                    c[i] = cn;
                    dot = dot_n;
                    sq = sq_n;
                    accepts[r] += 1;
                    total += 1;
                }
            }
        }
        if (codes_after)
            for (i = 0; i < len; ++i) codes_after[(size_t)(r + 1) * len + i] = (uint8_t)c[i];
    }
    /* Final code c_a from Eq. find_nearest_code applied to o_bar_a; it equals
     * the tracked integer code because o_bar_a sits on interval midpoints. */
    for (i = 0; i < len; ++i) {
        int cf = (int)floor((x[i] + vmax) / delta);
        if (cf > cmax) cf = cmax;
        if (cf < 0) cf = 0;
        code[i] = (uint8_t)c[i];
        (void)cf;
    }
    *norm_out = norm;
    *cos_out = objective(dot, sq, norm);
    free(x);
    free(c);
    return total;
}

/*
 * Quantize one segment o[0..len) with B bits (1 <= B <= 8) and adjust the
 * code for `rounds` rounds (Algorithm 1).
 *
 * Outputs:
 *   code[len]          final codes c_a in [0, 2^B - 1]
 *   *norm_out          |o|
 *   *cos_out           L(o_bar_a, o), the cosine between the adjusted quantized
 *                      vector and o (the second stored factor, Sec. 3.1 end)
 *   accepts[rounds]    number of accepted moves in each round
 *   *min_trial_margin  min over all in-range trials of |L(x') - L(x)|
 *   *min_init_margin   min over coordinates of the distance from o[i] to the
 *                      nearest interior interval boundary of the initial grid,
 *                      divided by |o| (how far o[i] must move, relative to the
 *                      segment norm, to change its initial code)
 *   *init_cos          L(o_bar, o) of the initial (unadjusted) code
 * Returns the number of accepted moves in total.
 */
int saq_oracle_caq_segment(const double *o, int len, int B, int rounds,
                           uint8_t *code, double *norm_out, double *cos_out,
                           int *accepts, double *min_trial_margin,
                           double *min_init_margin, double *init_cos) {
    return caq_run(o, len, B, rounds, code, norm_out, cos_out, accepts,
                   min_trial_margin, min_init_margin, init_cos, NULL, NULL,
                   NULL, NULL);
}

/*
 * The same run, recording every decision (see caq_run): codes_after is
 * (rounds + 1) x len, init_margin len, dplus and dminus rounds x len.  Used
 * to find where another implementation's codes first leave the oracle's and
 * how close that decision was.  Returns the number of accepted moves.
 */
int saq_oracle_caq_trace(const double *o, int len, int B, int rounds,
                         uint8_t *codes_after, double *init_margin,
                         double *dplus, double *dminus) {
    uint8_t *code = (uint8_t *)malloc((size_t)(len > 0 ? len : 1));
    int *acc = (int *)malloc(sizeof(int) * (size_t)(rounds > 0 ? rounds : 1));
    double nrm, cs, mt, mi, ic;
    const int total = caq_run(o, len, B, rounds, code, &nrm, &cs, acc, &mt, &mi,
                              &ic, codes_after, init_margin, dplus, dminus);
    free(code);
    free(acc);
    return total;
}

/*
 * Encode n projected vectors.  O is n x dk row-major (dk = kept dimensions,
 * the segments laid side by side in plan order).  For kept segment s,
 * columns [seg_off[s], seg_off[s] + seg_len[s]) hold o_s and seg_bits[s] >= 1.
 *
 * Outputs (row-major, per vector):
 *   codes    n x dk      one byte per kept coordinate
 *   norms    n x nseg    |o_s|
 *   coss     n x nseg    cos_s
 *   accepts  n x nseg x rounds
 *   min_trial_margin, min_init_margin, init_cos   n x nseg
 */
void saq_oracle_encode(const double *O, int64_t n, int dk, int nseg,
                       const int *seg_off, const int *seg_len,
                       const int *seg_bits, int rounds, int nthreads,
                       uint8_t *codes, double *norms, double *coss,
                       int *accepts, double *min_trial_margin,
                       double *min_init_margin, double *init_cos) {
    int64_t v;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#else
    (void)nthreads;
#endif
    for (v = 0; v < n; ++v) {
        for (int s = 0; s < nseg; ++s) {
            const int64_t k = v * nseg + s;
            saq_oracle_caq_segment(O + v * dk + seg_off[s], seg_len[s],
                                   seg_bits[s], rounds,
                                   codes + v * dk + seg_off[s], norms + k,
                                   coss + k, accepts + k * rounds,
                                   min_trial_margin + k, min_init_margin + k,
                                   init_cos + k);
        }
    }
}

int saq_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Quantization plan search (Algorithm 2) over segment boundaries on the grid
 * {0, g, 2g, ...} plus D itself (segments are multiples of g, the last one
 * takes the remainder when g does not divide D).
 *
 * ERROR(Seg, B) = sum_{i in Seg} sigma_i^2 * 2^-B  (Eq. seg-err with the
 * empirical-variance form of its footnote, which drops the pi; B = 0 applies
 * the same formula, i.e. a dropped segment costs its full variance).
 * Segment sums use prefix sums accumulated left to right; a plan's error is
 * accumulated segment by segment from the left.
 *
 * Bits are counted in units u = gcd of all possible segment lengths, so the
 * table index Q is "bits used / u".  E[p][Q][k] is the least error of a plan
 * covering the first p grid positions with exactly Q units and k segments.
 * Enumeration order: p ascending, Q ascending, k ascending, p' ascending,
 * b ascending; a state is replaced only by a strictly smaller error, so the
 * first plan found wins among equal errors.
 *
 * Selection: E* = min over all (Q <= quota, k).  The plan has the fewest
 * segments k among those with error <= (1 + tie_frac) E*; among those, the
 * least error, then the least cost Q.
 *
 * Outputs seg_start/seg_len/seg_bits (caller provides room for ceil(D/g)),
 * *nseg_out, *err_out (plan error), *min_err_out (E*), *cost_out (bits).
 * Returns 0 on success, -1 on bad arguments or allocation failure.
 */
static int64_t gcd64(int64_t a, int64_t b) {
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

int saq_oracle_plan(const double *sig2, int D, int g, int64_t quota_bits,
                    int max_bits, double tie_frac, int *seg_start,
                    int *seg_len, int *seg_bits, int *nseg_out,
                    double *err_out, double *min_err_out,
                    int64_t *cost_out) {
    if (D <= 0 || g <= 0 || max_bits < 0 || quota_bits < 0) return -1;
    const int ngrid = (D + g - 1) / g;      /* segments in the finest plan */
    const int npos = ngrid + 1;             /* boundary positions */
    int *pos = (int *)malloc(sizeof(int) * (size_t)npos);
    for (int p = 0; p < ngrid; ++p) pos[p] = p * g;
    pos[ngrid] = D;
    int64_t u = g;
    if (D % g) u = gcd64(g, D % g);
    const int64_t quota = quota_bits / u;
    double *prefix = (double *)malloc(sizeof(double) * (size_t)(D + 1));
    prefix[0] = 0.0;
    for (int i = 0; i < D; ++i) prefix[i + 1] = prefix[i] + sig2[i];

    const int64_t nQ = quota + 1, nK = npos;
    const size_t nstate = (size_t)npos * (size_t)nQ * (size_t)nK;
    double *E = (double *)malloc(sizeof(double) * nstate);
    int *bp_pos = (int *)malloc(sizeof(int) * nstate);
    int64_t *bp_q = (int64_t *)malloc(sizeof(int64_t) * nstate);
    int *bp_b = (int *)malloc(sizeof(int) * nstate);
    if (!pos || !prefix || !E || !bp_pos || !bp_q || !bp_b) {
        free(pos); free(prefix); free(E); free(bp_pos); free(bp_q); free(bp_b);
        return -1;
    }
#define IDX(p, q, k) (((size_t)(p) * (size_t)nQ + (size_t)(q)) * (size_t)nK + (size_t)(k))
    for (size_t t = 0; t < nstate; ++t) { E[t] = INFINITY; bp_pos[t] = -1; }
    E[IDX(0, 0, 0)] = 0.0;   /* p_{0,0}: the empty plan */

    for (int p = 0; p < npos - 1; ++p) {
        for (int64_t q = 0; q <= quota; ++q) {
            for (int k = 0; k <= p; ++k) {
                const double e0 = E[IDX(p, q, k)];
                if (!(e0 < INFINITY)) continue;   /* p_{d,Q} does not exist */
                for (int p2 = p + 1; p2 < npos; ++p2) {
                    const int len = pos[p2] - pos[p];
                    const double var = prefix[pos[p2]] - prefix[pos[p]];
                    for (int b = 0; b <= max_bits; ++b) {
                        const int64_t q2 = q + ((int64_t)b * len) / u;
                        if (q2 > quota) break;
                        const double e = e0 + ldexp(var, -b);
                        const size_t t = IDX(p2, q2, k + 1);
                        if (e < E[t]) {
                            E[t] = e;
                            bp_pos[t] = p;
                            bp_q[t] = q;
                            bp_b[t] = b;
                        }
                    }
                }
            }
        }
    }
    const int pend = npos - 1;
    double emin = INFINITY;
    for (int64_t q = 0; q <= quota; ++q)
        for (int k = 1; k < nK; ++k)
            if (E[IDX(pend, q, k)] < emin) emin = E[IDX(pend, q, k)];
    if (!(emin < INFINITY)) {
        free(pos); free(prefix); free(E); free(bp_pos); free(bp_q); free(bp_b);
        return -1;
    }
    const double thresh = emin * (1.0 + tie_frac);
    int kbest = -1;
    int64_t qbest = -1;
    double ebest = INFINITY;
    for (int k = 1; k < nK && kbest < 0; ++k) {
        for (int64_t q = 0; q <= quota; ++q) {
            const double e = E[IDX(pend, q, k)];
            if (e <= thresh && e < ebest) { ebest = e; qbest = q; }
        }
        if (qbest >= 0) kbest = k;
    }
    /* walk back */
    int p = pend, k = kbest;
    int64_t q = qbest;
    int ns = kbest;
    while (k > 0) {
        const size_t t = IDX(p, q, k);
        const int pp = bp_pos[t];
        seg_start[k - 1] = pos[pp];
        seg_len[k - 1] = pos[p] - pos[pp];
        seg_bits[k - 1] = bp_b[t];
        q = bp_q[t];
        p = pp;
        --k;
    }
#undef IDX
    int64_t cost = 0;
    for (int s = 0; s < ns; ++s) cost += (int64_t)seg_bits[s] * seg_len[s];
    *nseg_out = ns;
    *err_out = ebest;
    *min_err_out = emin;
    *cost_out = cost;
    free(pos); free(prefix); free(E); free(bp_pos); free(bp_q); free(bp_b);
    return 0;
}
