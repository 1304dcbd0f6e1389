// k_estimate.cu -- distance estimation from codes (Sec. 2.2 Eq. 3, Sec. 3.2
// Eq. estimator_inner_product, progressive prefixes of Sec. 3.2).
//
// Per kept segment s of vector v and query q (q_s = W_s (q_r - c)):
//   est_s = |o_s| <u_s, q_s> / (|u_s| cos_s),   u_s = 2 c - (2^b - 1)
// i.e. <o_bar_a, q> / <o_bar_a, o> |o|^2 with o_bar_a proportional to u_s
// (Delta <c, q> + q_sum (Delta/2 - v_max) = (Delta/2) <u, q>).
// d2 = |o_r - c|^2 + |q_r - c|^2 - 2 sum_s est_s.
// With a b-bit prefix the code is floor(c / 2^(B-b)) = the first b planes.
#include "saq_internal.h"

namespace saq {

namespace {

struct SegDesc {
    int off, len, bits, words, fidx;
    long long code_off;
};
constexpr int kMaxSeg = 64;
struct SegTable {
    SegDesc s[kMaxSeg];
};

__device__ __forceinline__ int decode(const uint64_t *planes, int words, int b, int j) {
    int c = 0;
    for (int p = 0; p < b; ++p) c = (c << 1) | (int)((planes[p * words + (j >> 6)] >> (j & 63)) & 1ull);
    return c;
}

// vscale[v * nk + s] = |o_s| / (|u_s| cos_s)  (0 for an all-zero segment)
__global__ void k_vec_scale(const uint8_t *__restrict__ codes, int64_t code_stride,
                            const float *__restrict__ factors, int nf, int64_t n, int nk,
                            SegTable t, int prefix_bits, float *__restrict__ vscale) {
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;
    for (int s = 0; s < nk; ++s) {
        const SegDesc g = t.s[s];
        const int b = (prefix_bits > 0 && prefix_bits < g.bits) ? prefix_bits : g.bits;
        const uint64_t *pl = reinterpret_cast<const uint64_t *>(codes + v * code_stride + g.code_off);
        float S = 0.f;
        for (int j = lane; j < g.len; j += 32) {
            const float u = (float)(2 * decode(pl, g.words, b, j) - ((1 << b) - 1));
            S = fmaf(u, u, S);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(0xffffffffu, S, off);
        if (lane == 0) {
            const float nrm = factors[v * nf + g.fidx];
            const float cs = factors[v * nf + g.fidx + 1];
            vscale[v * nk + s] = nrm > 0.f ? nrm / (sqrtf(S) * cs) : 0.f;
        }
    }
}

// one warp per (query, vector)
__global__ void k_estimate(const uint8_t *__restrict__ codes, int64_t code_stride,
                           const float *__restrict__ factors, int nf, int64_t n, int nk,
                           SegTable t, int prefix_bits, const float *__restrict__ vscale,
                           const float *__restrict__ qrot, int dk, const float *__restrict__ qn2,
                           int64_t nq, float *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n * nq) return;
    const int64_t q = w / n, v = w % n;
    const float *qr = qrot + q * dk;
    float est = 0.f;
    for (int s = 0; s < nk; ++s) {
        const SegDesc g = t.s[s];
        const int b = (prefix_bits > 0 && prefix_bits < g.bits) ? prefix_bits : g.bits;
        const uint64_t *pl = reinterpret_cast<const uint64_t *>(codes + v * code_stride + g.code_off);
        float acc = 0.f;
        for (int j = lane; j < g.len; j += 32) {
            const float u = (float)(2 * decode(pl, g.words, b, j) - ((1 << b) - 1));
            acc = fmaf(u, qr[g.off + j], acc);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        est = fmaf(acc, vscale[v * nk + s], est);
    }
    if (lane == 0) dist[q * n + v] = factors[v * nf] + qn2[q] - 2.f * est;
}

}  // namespace

saq_status launch_estimate(const saq_model *m, const uint8_t *codes, const float *factors,
                           int64_t n, const float *Qrot, const float *qn2, int64_t nq,
                           int prefix_bits, float *vscale, float *dist, cudaStream_t s) {
    const int nk = (int)m->kept.size();
    if (nk > kMaxSeg) return set_error(SAQ_ERR_UNSUPPORTED, "more than %d kept segments", kMaxSeg);
    SegTable t;
    for (int i = 0; i < nk; ++i) {
        const KeptSeg &k = m->kept[(size_t)i];
        t.s[i] = SegDesc{k.off, k.len, k.bits, k.words, k.fidx, (long long)k.code_off};
    }
    const int64_t cs = (int64_t)m->code_bytes;
    {
        LaunchTimer lt_(kKindOther, s);
        k_vec_scale<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(codes, cs, factors, m->nf, n, nk, t,
                                                             prefix_bits, vscale);
    }
    const int64_t warps = n * nq;
    {
        LaunchTimer lt_(kKindOther, s);
        k_estimate<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(codes, cs, factors, m->nf, n, nk, t,
                                                               prefix_bits, vscale, Qrot, m->dk, qn2,
                                                               nq, dist);
    }
    note_launches(2);
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace saq
