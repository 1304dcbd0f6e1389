// k_fit.cu -- the fit (Sec. 4.1, Sec. 4.2, Sec. 5.1):
//   mean c and covariance (1/N) sum (x - c)(x - c)^T accumulated in FP64 on
//   the GPU; eigen-decomposition (cuSOLVER, FP64), sigma^2 descending with
//   each eigenvector signed so its largest-magnitude component is positive;
//   the plan by Algorithm 2; one seeded random orthonormal matrix per kept
//   segment (QR of a Gaussian matrix, columns signed by diag(R): Haar); and
//   W = blockdiag(R_s) V_kept^T.
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <math.h>

#include <algorithm>
#include <memory>

#include "saq_internal.h"

namespace saq {

namespace {

__global__ void k_colsum_partial(const float *__restrict__ X, int64_t n, int d, int nsplit,
                                 double *__restrict__ partial) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int sp = blockIdx.y;
    if (j >= d) return;
    const int64_t per = (n + nsplit - 1) / nsplit;
    const int64_t r0 = sp * per, r1 = min(n, r0 + per);
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) s += (double)X[i * d + j];
    partial[(int64_t)sp * d + j] = s;
}

__global__ void k_colsum_final(const double *__restrict__ partial, int d, int nsplit, int64_t n,
                               double *__restrict__ mean) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += partial[(int64_t)sp * d + j];
    mean[j] = s / (double)n;
}

// 64 x 64 tile of sum_i (x_i - c)_a (x_i - c)_b over one row split, for
// tile pairs ti <= tj.  256 threads, 4 x 4 outputs each.
constexpr int kT = 64, kR = 16;

__global__ void __launch_bounds__(256)
k_cov_partial(const float *__restrict__ X, int64_t n, int d, const double *__restrict__ mean,
              int ntile, int nsplit, double *__restrict__ partial) {
    int lin = blockIdx.x, ti = 0;
    while (lin >= ntile - ti) { lin -= ntile - ti; ++ti; }
    const int tj = ti + lin;
    const int sp = blockIdx.y;
    __shared__ double A[kR][kT + 1];
    __shared__ double Bt[kR][kT + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    const int64_t per = (n + nsplit - 1) / nsplit;
    const int64_t r0 = sp * per, r1 = min(n, r0 + per);
    for (int64_t base = r0; base < r1; base += kR) {
        for (int e = tid; e < kR * kT; e += 256) {
            const int rr = e / kT, cc = e % kT;
            const int64_t i = base + rr;
            const int a = ti * kT + cc, b = tj * kT + cc;
            double va = 0.0, vb = 0.0;
            if (i < r1) {
                if (a < d) va = (double)X[i * d + a] - mean[a];
                if (b < d) vb = (double)X[i * d + b] - mean[b];
            }
            A[rr][cc] = va;
            Bt[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < kR; ++rr) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = A[rr][ty + 16 * q];
                b[q] = Bt[rr][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = ti * kT + ty + 16 * p, b = tj * kT + tx + 16 * q;
            if (a < d && b < d) partial[((int64_t)sp * d + a) * d + b] = acc[p][q];
        }
}

__global__ void k_cov_final(const double *__restrict__ partial, int d, int nsplit, int64_t n,
                            double *__restrict__ cov) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)d * d) return;
    int a = (int)(e / d), b = (int)(e % d);
    if (a / kT > b / kT) { const int t = a; a = b; b = t; }
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += partial[((int64_t)sp * d + a) * d + b];
    cov[e] = s / (double)n;
}

__global__ void k_scale_cols(double *__restrict__ Q, int n, const double *__restrict__ sgn) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    Q[e] *= sgn[e / n];  // column-major: column e / n
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    template <class T> T *as() { return static_cast<T *>(p); }
};

}  // namespace

saq_status launch_mean_f64(const float *X, int64_t n, int d, double *mean, double *partial,
                           int nsplit, cudaStream_t s) {
    dim3 g((unsigned)((d + 127) / 128), (unsigned)nsplit);
    k_colsum_partial<<<g, 128, 0, s>>>(X, n, d, nsplit, partial);
    k_colsum_final<<<(unsigned)((d + 127) / 128), 128, 0, s>>>(partial, d, nsplit, n, mean);
    note_launches(2);
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status launch_cov_f64(const float *X, int64_t n, int d, const double *mean, double *cov,
                          double *partial, int nsplit, cudaStream_t s) {
    const int nt = (d + kT - 1) / kT;
    dim3 g((unsigned)(nt * (nt + 1) / 2), (unsigned)nsplit);
    k_cov_partial<<<g, 256, 0, s>>>(X, n, d, mean, nt, nsplit, partial);
    const int64_t e = (int64_t)d * d;
    k_cov_final<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(partial, d, nsplit, n, cov);
    note_launches(2);
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace saq

using namespace saq;

#define SOLVER_CHECK(call)                                                         \
    do {                                                                           \
        cusolverStatus_t e__ = (call);                                             \
        if (e__ != CUSOLVER_STATUS_SUCCESS)                                        \
            return set_error(SAQ_ERR_CUDA, "%s failed: status %d", #call, (int)e__); \
    } while (0)
#define BLAS_CHECK(call)                                                           \
    do {                                                                           \
        cublasStatus_t e__ = (call);                                               \
        if (e__ != CUBLAS_STATUS_SUCCESS)                                          \
            return set_error(SAQ_ERR_CUDA, "%s failed: status %d", #call, (int)e__); \
    } while (0)

namespace {
struct Handles {
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    ~Handles() {
        if (sol) cusolverDnDestroy(sol);
        if (blas) cublasDestroy(blas);
    }
};
}  // namespace

extern "C" saq_status saq_fit(const float *X_dev, int64_t n, int32_t d, const saq_params *p,
                              saq_model **out, void *stream) {
    clear_error();
    if (!out) return set_error(SAQ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!X_dev || !p) return set_error(SAQ_ERR_INVALID, "NULL X or params");
    if (n < 2 || d < 1) return set_error(SAQ_ERR_INVALID, "need n >= 2 and d >= 1");
    if (p->max_bits < 0 || p->max_bits > 8)
        return set_error(SAQ_ERR_INVALID, "max_bits %d outside 0..8", p->max_bits);
    if (!(p->avg_bits >= 0.0) || p->avg_bits > p->max_bits)
        return set_error(SAQ_ERR_INVALID, "avg_bits must be in [0, max_bits]");
    if (p->seg_granularity < 1) return set_error(SAQ_ERR_INVALID, "seg_granularity < 1");
    if (!(p->tie_frac >= 0.0)) return set_error(SAQ_ERR_INVALID, "tie_frac < 0");
    if (((uintptr_t)X_dev & 15u) != 0) return set_error(SAQ_ERR_INVALID, "X not 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;

    const int nt = (d + 63) / 64;
    const int tiles = nt * (nt + 1) / 2;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(64, 1200 / tiles));
    nsplit = (int)std::min<int64_t>(nsplit, std::max<int64_t>(1, n / 64));
    DevBuf dmean, dpart, dcov, deval, dinfo, dwork;
    SAQ_CUDA_CHECK(cudaMalloc(&dmean.p, sizeof(double) * d));
    SAQ_CUDA_CHECK(cudaMalloc(&dpart.p, sizeof(double) * (size_t)nsplit * d * (size_t)d));
    SAQ_CUDA_CHECK(cudaMalloc(&dcov.p, sizeof(double) * (size_t)d * d));
    SAQ_CUDA_CHECK(cudaMalloc(&deval.p, sizeof(double) * d));
    SAQ_CUDA_CHECK(cudaMalloc(&dinfo.p, sizeof(int)));
    saq_status st = launch_mean_f64(X_dev, n, d, dmean.as<double>(), dpart.as<double>(),
                                    nsplit, s);
    if (st != SAQ_OK) return st;
    st = launch_cov_f64(X_dev, n, d, dmean.as<double>(), dcov.as<double>(), dpart.as<double>(),
                        nsplit, s);
    if (st != SAQ_OK) return st;

    Handles h;
    SOLVER_CHECK(cusolverDnCreate(&h.sol));
    SOLVER_CHECK(cusolverDnSetStream(h.sol, s));
    BLAS_CHECK(cublasCreate(&h.blas));
    BLAS_CHECK(cublasSetStream(h.blas, s));
    int lwork = 0;
    SOLVER_CHECK(cusolverDnDsyevd_bufferSize(h.sol, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, d, dcov.as<double>(), d,
                                             deval.as<double>(), &lwork));
    SAQ_CUDA_CHECK(cudaMalloc(&dwork.p, sizeof(double) * (size_t)std::max(1, lwork)));
    SOLVER_CHECK(cusolverDnDsyevd(h.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, d,
                                  dcov.as<double>(), d, deval.as<double>(), dwork.as<double>(),
                                  lwork, dinfo.as<int>()));
    std::vector<double> mean((size_t)d), ev((size_t)d), V((size_t)d * d);
    int info = 0;
    SAQ_CUDA_CHECK(cudaMemcpyAsync(mean.data(), dmean.p, sizeof(double) * d,
                                   cudaMemcpyDeviceToHost, s));
    SAQ_CUDA_CHECK(cudaMemcpyAsync(ev.data(), deval.p, sizeof(double) * d,
                                   cudaMemcpyDeviceToHost, s));
    SAQ_CUDA_CHECK(cudaMemcpyAsync(V.data(), dcov.p, sizeof(double) * (size_t)d * d,
                                   cudaMemcpyDeviceToHost, s));
    SAQ_CUDA_CHECK(cudaMemcpyAsync(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAQ_CUDA_CHECK(cudaStreamSynchronize(s));
    if (info != 0) return set_error(SAQ_ERR_CUDA, "eigen-decomposition failed (info %d)", info);

    // Sort descending (the solver returns ascending), canonical signs.
    std::vector<double> sig2((size_t)d), Vs((size_t)d * d);
    for (int k = 0; k < d; ++k) {
        const int src = d - 1 - k;
        sig2[(size_t)k] = std::max(0.0, ev[(size_t)src]);
        const double *col = &V[(size_t)src * d];
        int arg = 0;
        double best = -1.0;
        for (int i = 0; i < d; ++i)
            if (fabs(col[i]) > best) { best = fabs(col[i]); arg = i; }
        const double sg = col[arg] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < d; ++i) Vs[(size_t)k * d + i] = sg * col[i];
    }

    std::vector<saq_segment> plan;
    double perr = 0, pmin = 0;
    const int64_t quota = (int64_t)llround(p->avg_bits * d);
    if (plan_search(sig2.data(), d, p->seg_granularity, quota, p->max_bits, p->tie_frac, plan,
                    &perr, &pmin) != 0)
        return set_error(SAQ_ERR_OOM, "plan search failed (table too large?)");

    int64_t dk = 0;
    for (auto &sg : plan) if (sg.bits > 0) dk += sg.len;
    std::vector<double> W((size_t)(dk * d));
    if (dk > 0) {
        DevBuf dV, dG, dtau, dW, dsgn, dwork2;
        int maxlen = 0;
        for (auto &sg : plan) if (sg.bits > 0) maxlen = std::max(maxlen, sg.len);
        SAQ_CUDA_CHECK(cudaMalloc(&dV.p, sizeof(double) * (size_t)d * d));
        SAQ_CUDA_CHECK(cudaMemcpyAsync(dV.p, Vs.data(), sizeof(double) * (size_t)d * d,
                                       cudaMemcpyHostToDevice, s));
        SAQ_CUDA_CHECK(cudaMalloc(&dG.p, sizeof(double) * (size_t)maxlen * maxlen));
        SAQ_CUDA_CHECK(cudaMalloc(&dtau.p, sizeof(double) * (size_t)maxlen));
        SAQ_CUDA_CHECK(cudaMalloc(&dsgn.p, sizeof(double) * (size_t)maxlen));
        SAQ_CUDA_CHECK(cudaMalloc(&dW.p, sizeof(double) * (size_t)maxlen * d));
        int lw1 = 0, lw2 = 0;
        SOLVER_CHECK(cusolverDnDgeqrf_bufferSize(h.sol, maxlen, maxlen, dG.as<double>(), maxlen,
                                                 &lw1));
        SOLVER_CHECK(cusolverDnDorgqr_bufferSize(h.sol, maxlen, maxlen, maxlen, dG.as<double>(),
                                                 maxlen, dtau.as<double>(), &lw2));
        const int lw = std::max(1, std::max(lw1, lw2));
        SAQ_CUDA_CHECK(cudaMalloc(&dwork2.p, sizeof(double) * (size_t)lw));
        std::vector<double> G, diag, Wt;
        int row = 0, kidx = 0;
        for (auto &sg : plan) {
            if (sg.bits == 0) continue;
            const int L = sg.len;
            G.assign((size_t)L * L, 0.0);
            philox_gaussian(p->seed, (uint64_t)kidx, G.data(), G.size());
            SAQ_CUDA_CHECK(cudaMemcpyAsync(dG.p, G.data(), sizeof(double) * G.size(),
                                           cudaMemcpyHostToDevice, s));
            SOLVER_CHECK(cusolverDnDgeqrf(h.sol, L, L, dG.as<double>(), L, dtau.as<double>(),
                                          dwork2.as<double>(), lw, dinfo.as<int>()));
            // signs of diag(R) before orgqr overwrites the factor
            diag.assign((size_t)L, 0.0);
            SAQ_CUDA_CHECK(cudaMemcpy2DAsync(diag.data(), sizeof(double), dG.p,
                                             sizeof(double) * (L + 1), sizeof(double), L,
                                             cudaMemcpyDeviceToHost, s));
            SAQ_CUDA_CHECK(cudaStreamSynchronize(s));
            for (int i = 0; i < L; ++i) diag[(size_t)i] = diag[(size_t)i] < 0 ? -1.0 : 1.0;
            SAQ_CUDA_CHECK(cudaMemcpyAsync(dsgn.p, diag.data(), sizeof(double) * L,
                                           cudaMemcpyHostToDevice, s));
            SOLVER_CHECK(cusolverDnDorgqr(h.sol, L, L, L, dG.as<double>(), L, dtau.as<double>(),
                                          dwork2.as<double>(), lw, dinfo.as<int>()));
            const int64_t e = (int64_t)L * L;
            k_scale_cols<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(dG.as<double>(), L,
                                                                     dsgn.as<double>());
            note_launches();
            SAQ_CUDA_CHECK(cudaGetLastError());
            // W_s (L x d, column-major) = R_s (L x L) * V_s^T, V_s = columns [start, start+L)
            const double one = 1.0, zero = 0.0;
            BLAS_CHECK(cublasDgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_T, L, d, L, &one,
                                   dG.as<double>(), L, dV.as<double>() + (size_t)sg.start * d,
                                   d, &zero, dW.as<double>(), L));
            Wt.assign((size_t)L * d, 0.0);
            SAQ_CUDA_CHECK(cudaMemcpyAsync(Wt.data(), dW.p, sizeof(double) * Wt.size(),
                                           cudaMemcpyDeviceToHost, s));
            SAQ_CUDA_CHECK(cudaStreamSynchronize(s));
            for (int r = 0; r < L; ++r)
                for (int j = 0; j < d; ++j)
                    W[(size_t)(row + r) * d + j] = Wt[(size_t)j * L + r];
            row += L;
            ++kidx;
        }
    }
    st = saq_model_create(d, mean.data(), W.data(), plan.data(), (int32_t)plan.size(),
                          sig2.data(), p, out);
    if (st != SAQ_OK || dk == 0) return st;
    // the PCA directions of the kept dimensions, for the Sec. 4.3 bounds
    std::vector<double> Vt((size_t)(dk * d));
    int64_t row = 0;
    for (auto &sg : plan) {
        if (sg.bits == 0) continue;
        for (int r = 0; r < sg.len; ++r, ++row)
            std::copy(&Vs[(size_t)(sg.start + r) * d], &Vs[(size_t)(sg.start + r) * d] + d,
                      &Vt[(size_t)row * d]);
    }
    st = saq_model_set_basis(*out, Vt.data());
    if (st != SAQ_OK) {
        saq_model_free(*out);
        *out = nullptr;
    }
    return st;
}
