// saq_internal.h -- declarations shared by the library's translation units.
// Library-internal: nothing here is part of the C ABI in include/saq.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "saq.h"

namespace saq {

// ---------------------------------------------------------------- errors
saq_status set_error(saq_status s, const char *fmt, ...);
// Count `k` kernel launches (saq_kernel_launch_count).
void note_launches(int k = 1);

// Optional per-launch device timing (saq_kernel_timing): a scope that records
// a CUDA event on `s` when it is opened (just before a launch) and another
// when it closes (just after it).
enum KernelKind { kKindProject = 0, kKindQuantize = 1, kKindOther = 2, kKindCount = 3 };
struct LaunchTimer {
    LaunchTimer(int kind, cudaStream_t s);
    ~LaunchTimer();
    LaunchTimer(const LaunchTimer &) = delete;
    LaunchTimer &operator=(const LaunchTimer &) = delete;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
};
void clear_error();

#define SAQ_CUDA_CHECK(call)                                                   \
    do {                                                                       \
        cudaError_t e__ = (call);                                              \
        if (e__ != cudaSuccess)                                                \
            return ::saq::set_error(SAQ_ERR_CUDA, "%s failed: %s (%s:%d)",     \
                                    #call, cudaGetErrorString(e__), __FILE__,  \
                                    __LINE__);                                 \
    } while (0)

// ------------------------------------------------------------------ model
// A kept segment in the projected (kept-column) space.
struct KeptSeg {
    int32_t start;     // first PCA dimension of the segment
    int32_t off;       // first column of the segment in O (kept space)
    int32_t len;       // coordinates
    int32_t bits;      // 1..8
    int64_t code_off;  // byte offset of the segment inside a code record
    int32_t words;     // 64-bit words per bit-plane = ceil(len / 64)
    int32_t fidx;      // factor index of |o_s| (cos_s follows)
};

// Device operands of the tensor-core projection (built per precision).
struct TcOperands {
    int precision = -1;
    void *w_hi = nullptr;     // dk_pad x d_pad, cut into (pass, K block) tiles (FP16 hi / BF16 / FP8)
    void *w_lo = nullptr;     // the same for the FP16 lo part, or nullptr
    float *col_scale = nullptr;  // per output column dequant scale (dk_pad)
    int dk_pad = 0;
    int d_pad = 0;
    void *extra = nullptr;    // tensor maps, padded mean, error word (k_tc.cu)
};

// Column ends of the kept segments in the projected (kept) space, for the
// per-(row, segment) v_max of the projection epilogue.
struct SegCols {
    int32_t end[64];
    int32_t nk;
};

}  // namespace saq

struct saq_model {
    int32_t d = 0;
    int32_t dk = 0;           // kept dimensions
    int32_t rounds = 6;
    int32_t precision = SAQ_PREC_FP32;
    int device = 0;
    std::vector<saq_segment> plan;        // all segments
    std::vector<saq::KeptSeg> kept;       // kept segments, plan order
    std::vector<double> mean;             // d
    std::vector<double> W;                // dk x d row-major
    std::vector<double> sig2;             // d (zeros if unknown)
    std::vector<double> Vt;               // dk x d PCA directions of the kept dims (empty if unknown)
    size_t code_bytes = 0;
    int32_t nf = 1;                       // factors per vector
    // device copies
    float *d_mean = nullptr;              // d
    float *d_W = nullptr;                 // dk x d FP32 row-major
    float *d_B = nullptr;                 // dk x d FP32: row i = sigma_i v_i^T (if Vt is known)
    saq::TcOperands tc;
};

namespace saq {

// ------------------------------------------------------------ host pieces
// Algorithm 2 plan search (library implementation).
int plan_search(const double *sig2, int D, int g, int64_t quota_bits,
                int max_bits, double tie_frac, std::vector<saq_segment> &out,
                double *err, double *min_err);

// Counter-based Gaussian draws (Philox4x32-10 + Box-Muller), FP64.
void philox_gaussian(uint64_t seed, uint64_t stream_id, double *out, size_t n);

saq_status model_finalize(saq_model *m);  // derive kept segs, upload
// Stream-ordered scratch from the library's own pool on the current device
// (kept cached up to kPoolKeepBytes between calls); free with cudaFreeAsync.
constexpr size_t kPoolKeepBytes = (size_t)8 << 30;
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
saq_status model_upload_basis(saq_model *m);  // d_B from Vt and sig2
saq_status model_build_tc(saq_model *m, int precision, cudaStream_t s);
void model_release_device(saq_model *m);

// ---------------------------------------------------------------- kernels
// Models per grouped launch (a serving batch of several collections).
constexpr int kMaxGroups = 4;
// Layout of projected rows: row-major (ldo floats per row) or interleaved by
// groups of 32 rows, O_i[((row / 32) * dk + col) * 32 + row % 32] (the layout
// the quantize kernel reads; ldo is ignored).
enum { kRowMajor = 0, kInterleaved = 1 };
// O[i, :] = W (x_i - c) for rows [0, n): FP32 SIMT GEMM, exact FP32 products.
saq_status launch_project_simt(const saq_model *m, const float *X, int64_t n,
                               float *O, int64_t ldo, int layout, cudaStream_t s);
// Tensor-core projection (tcgen05 + TMA); precision from m->tc.  With the
// interleaved layout and vmax != NULL it also writes, per row and kept
// segment, max |o| into vmax (interleaved like O: [(row/32) * nk + s] * 32 +
// row % 32; the caller zeroes it first).
// err: the device error word the launch raises (bounded waits that gave up,
// input rows out of range); NULL selects the model's own word.
saq_status launch_project_tc(const saq_model *m, const float *X, int64_t n,
                             float *O, int64_t ldo, int layout, float *norms2,
                             int64_t norms_stride, float *vmax, int *err, cudaStream_t s);
SegCols seg_cols(const saq_model *m);
// One model's rows of a grouped projection launch (interleaved output, v_max
// zeroed by the caller, |x - c|^2 into norms[i * nstride]).
struct ProjJob {
    const saq_model *m;
    const float *X;
    int64_t n;
    float *O;
    float *norms;
    int64_t nstride;
    float *vmax;
    int *err;  // NULL: the model's own error word
};
// Up to kMaxGroups models of one tensor-core precision in one persistent
// launch whose CTAs take the tiles from the device work counter *queue
// (zero at launch).
saq_status launch_project_tc_grouped(const ProjJob *jobs, int njobs, int *queue, cudaStream_t s);
bool tc_supported(const saq_model *m);
void tc_release(saq_model *m);
// Reads and clears the model's device error word of the tensor-core
// projection (synchronises `s`): SAQ_ERR_TIMEOUT if a bounded wait gave up,
// SAQ_ERR_RANGE if an input row was out of range.
saq_status tc_check_error(const saq_model *m, cudaStream_t s);
// The status (and message) of a value read from an error word.
saq_status tc_error_status(int code);
// The model's own error word (NULL without tensor-core operands).
int *tc_error_word(const saq_model *m);
// norms2[i * stride] = |x_i - c|^2
saq_status launch_rownorm2(const saq_model *m, const float *X, int64_t n,
                           float *out, int64_t stride, cudaStream_t s);
// Strided copy of n floats.
saq_status launch_copy_strided(const float *src, int64_t sstride, float *dst,
                               int64_t dstride, int64_t n, cudaStream_t s);
// Quantize + adjust + pack every kept segment for rows [0, n) of interleaved
// projected rows Oi, with a byte scratch cs of the same layout (k_caq1.cu).
saq_status launch_caq1(const saq_model *m, const float *Oi, int64_t n, uint8_t *cs,
                       const float *vmax, uint8_t *codes, float *factors, cudaStream_t s);
// Several models' rows in one launch (a batch of several collections): each
// job as for launch_caq1.  At most kMaxGroups jobs.
struct CaqJob {
    const saq_model *m;
    const float *Oi;
    int64_t n;
    uint8_t *cs;
    const float *vmax;
    uint8_t *codes;
    float *factors;
};
// Up to kMaxGroups models in one persistent launch whose warps take their
// (model, segment, 32-row group) items from the device work counter *queue
// (zero at launch).
saq_status launch_caq1_grouped(const CaqJob *jobs, int njobs, int *queue, cudaStream_t s);
// vmax of every (row, kept segment) from interleaved rows Oi (k_caq1.cu).
// Lane-steps per second of the adjustment step on register-resident data
// (saq_quantize_step_ceiling).
saq_status step_ceiling(int warps_per_sm, int bits, double *lane_steps_per_s);
saq_status launch_seg_vmax(const saq_model *m, const float *Oi, int64_t n, float *vmax,
                           cudaStream_t s);
// Row-major O -> interleaved Oi.
saq_status launch_interleave(const float *O, int64_t ldo, int64_t n, int dk, float *Oi,
                             cudaStream_t s);
// Scratch of an encode of up to `rows` rows: the interleaved projected rows
// (FP32) followed by the byte code scratch (saq_encode.cu).
size_t encode_scratch_bytes(const saq_model *m, int64_t rows);
// Projection of rows [0, n) (saq_encode.cu); vmax as for launch_project_tc
// (may be NULL).
saq_status project_rows(const saq_model *m, const float *X, int64_t n, float *O, int64_t ldo,
                        int layout, float *norms, int64_t nstride, float *vmax, cudaStream_t s,
                        int *err = nullptr);
// Quantization of rows [0, n) from interleaved projected rows in `scratch`.
saq_status quantize_rows(const saq_model *m, void *scratch, int64_t rows_cap, int64_t n,
                         uint8_t *codes, float *factors, cudaStream_t s);
// The whole encode of rows [0, n) with a scratch for `rows` rows.
// err as for launch_project_tc.
saq_status encode_rows(const saq_model *m, const float *X, int64_t n, uint8_t *codes,
                       float *factors, void *scratch, int64_t rows, cudaStream_t s,
                       int *err = nullptr);
// 1 if the model's encode runs the tensor-core projection.
bool use_tc(const saq_model *m);
// One model's rows of a grouped encode: n <= the rows its scratch holds
// (encode_scratch_bytes(m, n) bytes).
struct EncodeJob {
    const saq_model *m;
    const float *X;
    int64_t n;
    uint8_t *codes;
    float *factors;
    void *scratch;
};
// The encode of up to kMaxGroups models' rows with one persistent projection
// launch and one persistent quantize launch; every model with kept
// dimensions must use the tensor-core projection, all in one precision.  err
// as for launch_project_tc; queue: two device ints, the launches' work
// counters (zeroed here on s before the launches).
saq_status encode_grouped(const EncodeJob *jobs, int njobs, cudaStream_t s, int *err, int *queue);
// Estimator.
saq_status launch_estimate_staged(const saq_model *m, const uint8_t *codes, const float *factors,
                                  int64_t n, const float *Q, const float *Qrot, const float *qn2,
                                  int64_t nq, float m_conf, float *vscale, float *qsig,
                                  float *bounds, cudaStream_t s);
saq_status launch_estimate(const saq_model *m, const uint8_t *codes,
                           const float *factors, int64_t n, const float *Qrot,
                           const float *qn2, int64_t nq, int prefix_bits,
                           float *vscale, float *dist, cudaStream_t s);
// Fit kernels (FP64).
saq_status launch_mean_f64(const float *X, int64_t n, int d, double *mean,
                           double *partial, int nsplit, cudaStream_t s);
saq_status launch_cov_f64(const float *X, int64_t n, int d, const double *mean,
                          double *cov, double *partial, int nsplit,
                          cudaStream_t s);

}  // namespace saq
