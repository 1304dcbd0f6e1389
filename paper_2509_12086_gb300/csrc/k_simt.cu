// k_simt.cu -- CUDA-core kernels of the projection step:
//   * the FP32 projection O = (X - c) W^T (Sec. 3.1 Eq. rotate with the
//     combined PCA + segment-rotation matrix of Sec. 5.1), exact FP32
//     products accumulated in k order; the reference-grade path and the
//     query-rotation path of the estimator;
//   * |x - c|^2 per row (the norm factor of Eq. 3);
//   * a strided copy.
#include "saq_internal.h"

namespace saq {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 8;

__global__ void __launch_bounds__(256)
k_project_simt(const float *__restrict__ X, int64_t n, int d,
               const float *__restrict__ c, const float *__restrict__ W, int dk,
               float *__restrict__ O, int64_t ldo, int il) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    const int col0 = blockIdx.y * kBN;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int lr = tid >> 1;          // tile row / column this thread loads
    const int lk = (tid & 1) * 4;     // first of its 4 k positions
    for (int k0 = 0; k0 < d; k0 += kBK) {
        const int64_t gi = row0 + lr;
        const int gj = col0 + lr;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + lk + q;
            float a = 0.f, b = 0.f;
            if (gi < n && k < d) a = X[gi * d + k] - c[k];
            if (gj < dk && k < d) b = W[(int64_t)gj * d + k];
            As[lk + q][lr] = a;
            Bs[lk + q][lr] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gi = row0 + ty + 16 * i;
        if (gi >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gj = col0 + tx + 16 * j;
            if (gj < dk) {
                if (il) O[(((gi >> 5) * dk + gj) << 5) + (gi & 31)] = acc[i][j];
                else O[gi * ldo + gj] = acc[i][j];
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_rownorm2(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ c,
           float *__restrict__ out, int64_t stride) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float *x = X + row * d;
    float s = 0.f;
    for (int k = lane; k < d; k += 32) {
        const float y = x[k] - c[k];
        s = fmaf(y, y, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[row * stride] = s;
}

__global__ void k_copy_strided(const float *__restrict__ src, int64_t ss,
                               float *__restrict__ dst, int64_t ds, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i * ds] = src[i * ss];
}

}  // namespace

saq_status launch_project_simt(const saq_model *m, const float *X, int64_t n,
                               float *O, int64_t ldo, int layout, cudaStream_t s) {
    if (n <= 0 || m->dk <= 0) return SAQ_OK;
    // kBM * 65535 is a multiple of 32, so interleaved chunks start on a group
    for (int64_t r0 = 0; r0 < n; r0 += (int64_t)kBM * 65535) {
        const int64_t rows = n - r0 < (int64_t)kBM * 65535 ? n - r0 : (int64_t)kBM * 65535;
        dim3 grid((unsigned)((rows + kBM - 1) / kBM), (unsigned)((m->dk + kBN - 1) / kBN));
        float *Ob = layout == kInterleaved ? O + r0 * m->dk : O + r0 * ldo;
        {
            LaunchTimer lt_(kKindProject, s);
            k_project_simt<<<grid, 256, 0, s>>>(X + r0 * m->d, rows, m->d, m->d_mean, m->d_W,
                                                m->dk, Ob, ldo, layout == kInterleaved ? 1 : 0);
        }
        note_launches();
    }
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status launch_rownorm2(const saq_model *m, const float *X, int64_t n,
                           float *out, int64_t stride, cudaStream_t s) {
    if (n <= 0) return SAQ_OK;
    const int64_t blocks = (n + 7) / 8;
    {
        LaunchTimer lt_(kKindOther, s);
        k_rownorm2<<<(unsigned)blocks, 256, 0, s>>>(X, n, m->d, m->d_mean, out, stride);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status launch_copy_strided(const float *src, int64_t sstride, float *dst,
                               int64_t dstride, int64_t n, cudaStream_t s) {
    if (n <= 0) return SAQ_OK;
    {
        LaunchTimer lt_(kKindOther, s);
        k_copy_strided<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, sstride, dst, dstride, n);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace saq
