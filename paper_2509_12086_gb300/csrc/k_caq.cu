// k_caq.cu -- quantize, adjust and pack one kept segment (Sec. 3.1,
// Eq. find_nearest_code, Eq. adj-obj, Algorithm 1; Sec. 4.2 "quantize each
// segment separately").
//
// One warp per (vector, segment).  Lane l holds coordinates m*32 + l of the
// segment in registers (o and the code in half-step units u = 2c - (2^B-1)),
// for m < NCH.  Algorithm 1 is a sequential scan; the warp runs it exactly:
// every lane of the current 32-coordinate chunk tests its coordinate against
// the current state, a ballot finds the first coordinate (in scan order) with
// an improving move, that move is applied, and the coordinates after it are
// tested again against the new state.  Coordinates before the first accepted
// one were tested against the state they would have seen, so the result is
// the paper's order.  Per coordinate +Delta is tried before -Delta; at most
// one of the two can raise the cosine (the set {x : cos(x, o) > L} is a
// convex cone for L > 0, so a line meets it in an interval), and after an
// accepted +Delta the paper's -Delta trial returns to the old point and is
// always rejected.
//
// Decision in closed form: with I = <u, o> > 0 and S = |u|^2 (exact integer),
// moving u_i by 2s (s = +-1) raises I/sqrt(S) iff
//     s*o_i*alpha + o_i^2*beta > s*u_i + 1,   alpha = S/I, beta = S/I^2,
// (square both sides of I'/sqrt(S') > I/sqrt(S); the moves that could make
// I' <= 0 are never improving).  Both sides are first-order quantities, so
// FP32 decides correctly down to relative cosine margins far below 1e-7.
// I and S are recomputed exactly at the start of every round; within a
// round the eligible lanes of a chunk are a uniform bit mask ANDed into the
// ballot, and the two thresholds of the current chunk (u+1, 1-u, or +inf at
// the edge of the grid) are kept in registers, so a pass without a move costs
// a handful of instructions and each accepted move one shuffle-and-update.
#include "saq_internal.h"

namespace saq {

namespace {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}
__device__ __forceinline__ int warp_sum_i(int x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}
__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, off));
    return x;
}

template <int NCH>
__global__ void __launch_bounds__(256, (NCH >= 24) ? 1 : 2)
k_caq(const float *__restrict__ O, int64_t ldo, int64_t n, int col, int len, int B,
      int rounds, uint8_t *__restrict__ codes, int64_t code_stride, int64_t code_off,
      int words, float *__restrict__ factors, int nf, int fidx) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;  // uniform per warp
    const float *orow = O + v * ldo + col;
    float o[NCH], u[NCH];
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
        const int j = m * 32 + lane;
        o[m] = (j < len) ? __ldg(orow + j) : 0.f;
    }
    float vmax = 0.f, n2 = 0.f;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
        vmax = fmaxf(vmax, fabsf(o[m]));
        n2 = fmaf(o[m], o[m], n2);
    }
    vmax = warp_max(vmax);
    n2 = warp_sum(n2);
    float *fout = factors + v * nf;
    uint64_t *cout = reinterpret_cast<uint64_t *>(codes + v * code_stride + code_off);
    if (vmax == 0.f) {
        // All-zero segment (the paper is silent): codes 0, |o| = 0, cos = 1.
        for (int t = lane; t < B * words; t += 32) cout[t] = 0ull;
        if (lane == 0) {
            fout[fidx] = 0.f;
            fout[fidx + 1] = 1.f;
        }
        return;
    }
    const int cmax = (1 << B) - 1;
    const float cmaxf = (float)cmax;
    // Eq. find_nearest_code: c = floor((o + v_max) / Delta), Delta = 2 v_max / 2^B
    const float inv_delta = (float)(1 << (B - 1)) / vmax;
    int S = 0;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
        const int j = m * 32 + lane;
        int ui = 0;
        if (j < len) {
            int c = (int)floorf((o[m] + vmax) * inv_delta);
            c = c < 0 ? 0 : (c > cmax ? cmax : c);
            ui = 2 * c - cmax;
        }
        u[m] = (float)ui;
        S += ui * ui;
    }
    S = warp_sum_i(S);
    float Sf = (float)S;

    const float kInf = __int_as_float(0x7f800000);
    for (int r = 0; r < rounds; ++r) {
        // exact state at the start of the round
        float I = 0.f;
        int Si = 0;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            I = fmaf(u[m], o[m], I);
            Si += (int)u[m] * (int)u[m];
        }
        I = warp_sum(I);
        Sf = (float)warp_sum_i(Si);
        float rI = __fdividef(1.f, I);
        float alpha = Sf * rI;
        float beta = alpha * rI;
        bool moved = false;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            if (m * 32 >= len) break;
            const float om = o[m];
            const float o2 = om * om;
            // thresholds of the two moves; +inf where the move leaves the grid
            // (padding lanes have o = u = 0 and never pass them)
            float up1 = u[m] < cmaxf ? u[m] + 1.f : kInf;
            float um1 = u[m] > -cmaxf ? 1.f - u[m] : kInf;
            unsigned eligible = 0xffffffffu;
            while (true) {
                const float t = o2 * beta;
                const bool ap = fmaf(om, alpha, t) > up1;
                const bool am = fmaf(-om, alpha, t) > um1;
                const unsigned mask = __ballot_sync(0xffffffffu, ap || am) & eligible;
                if (mask == 0u) break;
                const int p = __ffs(mask) - 1;
                const bool plus = (__ballot_sync(0xffffffffu, ap) >> p) & 1u;
                const float sgn = plus ? 1.f : -1.f;
                const float op = __shfl_sync(0xffffffffu, om, p);
                const float up = __shfl_sync(0xffffffffu, u[m], p);
                I = fmaf(2.f * sgn, op, I);
                Sf += fmaf(4.f * sgn, up, 4.f);
                rI = __fdividef(1.f, I);
                alpha = Sf * rI;
                beta = alpha * rI;
                if (lane == p) {
                    const float un = up + 2.f * sgn;
                    u[m] = un;
                    up1 = un < cmaxf ? un + 1.f : kInf;
                    um1 = un > -cmaxf ? 1.f - un : kInf;
                }
                eligible = (p == 31) ? 0u : (0xfffffffeu << p);
                moved = true;
            }
        }
        if (!moved) break;  // a round without a move leaves the state unchanged
    }
    {
        int Si = 0;
#pragma unroll
        for (int m = 0; m < NCH; ++m) Si += (int)u[m] * (int)u[m];
        Sf = (float)warp_sum_i(Si);
    }

    float I = 0.f;
#pragma unroll
    for (int m = 0; m < NCH; ++m) I = fmaf(u[m], o[m], I);
    I = warp_sum(I);
    const float nrm = sqrtf(n2);
    if (lane == 0) {
        fout[fidx] = nrm;
        fout[fidx + 1] = I / (sqrtf(Sf) * nrm);
    }
    // Bit-planes, most significant first; 64-bit little-endian words.
    for (int p = 0; p < B; ++p) {
        const int bit = B - 1 - p;
#pragma unroll
        for (int m = 0; m < NCH; m += 2) {
            if (m * 32 >= len) break;
            const int c0 = ((int)(u[m] + cmaxf)) >> 1;
            const bool b0 = (m * 32 + lane < len) && ((c0 >> bit) & 1);
            const unsigned w0 = __ballot_sync(0xffffffffu, b0);
            unsigned w1 = 0u;
            if (m + 1 < NCH) {
                const int c1 = ((int)(u[m + 1] + cmaxf)) >> 1;
                const bool b1 = ((m + 1) * 32 + lane < len) && ((c1 >> bit) & 1);
                w1 = __ballot_sync(0xffffffffu, b1);
            }
            const int word = p * words + m / 2;
            if (lane == (word & 31)) cout[word] = (uint64_t)w0 | ((uint64_t)w1 << 32);
        }
    }
}

template <int NCH>
void launch(const float *O, int64_t ldo, int64_t n, const KeptSeg &k, int rounds,
            uint8_t *codes, int64_t cs, float *factors, int nf, cudaStream_t s) {
    const int64_t blocks = (n + 7) / 8;
    k_caq<NCH><<<(unsigned)blocks, 256, 0, s>>>(O, ldo, n, k.off, k.len, k.bits, rounds, codes,
                                                cs, k.code_off, k.words, factors, nf, k.fidx);
    note_launches();
}

}  // namespace

saq_status launch_caq_segment(const saq_model *m, int seg, const float *O, int64_t ldo,
                              int64_t n, uint8_t *codes, float *factors, cudaStream_t s) {
    if (n <= 0) return SAQ_OK;
    const KeptSeg &k = m->kept[(size_t)seg];
    const int nch = (k.len + 31) / 32;
    const int64_t cs = (int64_t)m->code_bytes;
    if (nch <= 2) launch<2>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 4) launch<4>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 6) launch<6>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 8) launch<8>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 12) launch<12>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 16) launch<16>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 24) launch<24>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else if (nch <= 32) launch<32>(O, ldo, n, k, m->rounds, codes, cs, factors, m->nf, s);
    else
        return set_error(SAQ_ERR_UNSUPPORTED,
                         "segment of %d coordinates exceeds the 1024 supported", k.len);
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace saq
