// k_estimate.cu -- distance estimation from codes (Sec. 2.2 Eq. 3, Sec. 3.2
// Eq. estimator_inner_product, progressive prefixes of Sec. 3.2).
//
// Per kept segment s of vector v and query q (q_s = W_s (q_r - c)):
//   est_s = |o_s| <u_s, q_s> / (|u_s| cos_s),   u_s = 2 c - (2^b - 1)
// i.e. <o_bar_a, q> / <o_bar_a, o> |o|^2 with o_bar_a proportional to u_s
// (Delta <c, q> + q_sum (Delta/2 - v_max) = (Delta/2) <u, q>).
// d2 = |o_r - c|^2 + |q_r - c|^2 - 2 sum_s est_s.
// With a b-bit prefix the code is floor(c / 2^(B-b)) = the first b planes.
//
// Multi-stage estimation (Sec. 4.3): the kept segments are taken in plan
// order (decreasing variance); after t stages the first t contribute est_s
// and each remaining one its Chebyshev bound m * sigma_Seg(q), where
// sigma_Seg(q)^2 = sum_{i in Seg} sigma_i^2 (v_i . (q_r - c))^2 is the
// variance of <o_seg, q_seg> over the data:
//   lb_t = |o_r - c|^2 + |q_r - c|^2 - 2 (sum_{s<t} est_s + m sum_{s>=t} sigma_s).
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

// sig[q * nk + s] = sigma_Seg(q) = |B_s (q_r - c)|, B_s = rows sigma_i v_i^T of
// the segment; one warp per (query, kept segment)
__global__ void k_query_sigma(const float *__restrict__ Q, int64_t nq, int d,
                              const float *__restrict__ mean, const float *__restrict__ B, int nk,
                              SegTable t, float *__restrict__ sig) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nq * nk) return;
    const int64_t q = w / nk;
    const int s = (int)(w % nk);
    const SegDesc g = t.s[s];
    const float *qv = Q + q * d;
    float acc = 0.f;
    for (int i = 0; i < g.len; ++i) {
        const float *b = B + (int64_t)(g.off + i) * d;
        float dot = 0.f;
        for (int k = lane; k < d; k += 32) dot = fmaf(b[k], qv[k] - mean[k], dot);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
        acc = fmaf(dot, dot, acc);
    }
    if (lane == 0) sig[q * nk + s] = sqrtf(acc);
}

// bounds[(q * n + v) * (nk + 1) + t] = lb_t; one warp per (query, vector)
__global__ void k_estimate_staged(const uint8_t *__restrict__ codes, int64_t code_stride,
                                  const float *__restrict__ factors, int nf, int64_t n, int nk,
                                  SegTable t, const float *__restrict__ vscale,
                                  const float *__restrict__ qrot, int dk,
                                  const float *__restrict__ qn2, int64_t nq,
                                  const float *__restrict__ qsig, float m_conf,
                                  float *__restrict__ bounds) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n * nq) return;
    const int64_t q = w / n, v = w % n;
    const float *qr = qrot + q * dk;
    const float *sg = qsig + q * nk;
    const float base = factors[v * nf] + qn2[q];
    float *out = bounds + (q * n + v) * (int64_t)(nk + 1);
    auto rest = [&](int t0) {  // m * sum_{s >= t0} sigma_s
        float r = 0.f;
        for (int s = t0; s < nk; ++s) r += sg[s];
        return m_conf * r;
    };
    if (lane == 0) out[0] = base - 2.f * rest(0);
    float done = 0.f;
    for (int s = 0; s < nk; ++s) {
        const SegDesc g = t.s[s];
        const uint64_t *pl = reinterpret_cast<const uint64_t *>(codes + v * code_stride + g.code_off);
        float acc = 0.f;
        for (int j = lane; j < g.len; j += 32) {
            const float u = (float)(2 * decode(pl, g.words, g.bits, j) - ((1 << g.bits) - 1));
            acc = fmaf(u, qr[g.off + j], acc);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        done = fmaf(acc, vscale[v * nk + s], done);
        if (lane == 0) out[s + 1] = base - 2.f * (done + rest(s + 1));
    }
}

SegTable seg_table(const saq_model *m) {
    SegTable t;
    for (size_t i = 0; i < m->kept.size(); ++i) {
        const KeptSeg &k = m->kept[i];
        t.s[i] = SegDesc{k.off, k.len, k.bits, k.words, k.fidx, (long long)k.code_off};
    }
    return t;
}

}  // namespace

saq_status launch_estimate_staged(const saq_model *m, const uint8_t *codes, const float *factors,
                                  int64_t n, const float *Q, const float *Qrot, const float *qn2,
                                  int64_t nq, float m_conf, float *vscale, float *qsig,
                                  float *bounds, cudaStream_t s) {
    const int nk = (int)m->kept.size();
    if (nk > kMaxSeg) return set_error(SAQ_ERR_UNSUPPORTED, "more than %d kept segments", kMaxSeg);
    const SegTable t = seg_table(m);
    const int64_t cs = (int64_t)m->code_bytes;
    {
        LaunchTimer lt_(kKindOther, s);
        k_vec_scale<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(codes, cs, factors, m->nf, n, nk, t, 0,
                                                             vscale);
    }
    {
        LaunchTimer lt_(kKindOther, s);
        k_query_sigma<<<(unsigned)((nq * nk + 7) / 8), 256, 0, s>>>(Q, nq, m->d, m->d_mean, m->d_B,
                                                                     nk, t, qsig);
    }
    {
        LaunchTimer lt_(kKindOther, s);
        k_estimate_staged<<<(unsigned)((n * nq + 7) / 8), 256, 0, s>>>(
            codes, cs, factors, m->nf, n, nk, t, vscale, Qrot, m->dk, qn2, nq, qsig, m_conf, bounds);
    }
    note_launches(3);
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

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
