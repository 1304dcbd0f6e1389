/*
 * saq.h -- C ABI of the GB300-native SAQ vector encoder.
 *
 * SAQ (Segmented CAQ, arXiv 2509.12086) maps each data vector o_r to a
 * compact code from which distances to query vectors can be estimated
 * (Sec. 1 problem statement; Sec. 2.2 Eq. 2-3).  The library implements the
 * fit (Sec. 4.1 PCA, Sec. 4.2 Algorithm 2, per-segment random rotations), the
 * encode hot path (Sec. 3.1 Eq. rotate, Eq. find_nearest_code, Algorithm 1,
 * Sec. 4.2 per-segment quantization, Sec. 5.1 combined PCA+rotation matrix)
 * and the distance estimator (Sec. 3.2 Eq. estimator_inner_product).
 *
 * Conventions for every entry point:
 *   - Plain pointers and sizes only.  "_dev" pointers are CUDA device
 *     pointers on the current device; "_host" pointers are host memory.
 *   - Device buffers passed in must be 16-byte aligned.
 *   - The caller owns every data buffer it passes; the library owns models.
 *   - Calls that take a `stream` (a cudaStream_t passed as void*, NULL for
 *     the legacy default stream) are asynchronous on that stream unless
 *     stated otherwise; buffers must stay valid until the stream reaches the
 *     call's work.
 *   - Errors are returned as saq_status; no exception crosses the ABI.
 *     Arguments are validated before any launch.  saq_last_error() returns a
 *     message for the calling thread's last failure.
 *   - A model may be used by one encode/estimate call at a time per stream;
 *     concurrent calls on different streams with the same model are allowed
 *     (the model is read-only during encode; scratch is stream-ordered).
 */
#ifndef SAQ_H
#define SAQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct saq_model saq_model;

typedef enum {
    SAQ_OK = 0,
    SAQ_ERR_INVALID = 1,     /* bad argument; nothing was launched          */
    SAQ_ERR_CUDA = 2,        /* a CUDA runtime / library call failed        */
    SAQ_ERR_OOM = 3,         /* device or host allocation failed            */
    SAQ_ERR_TIMEOUT = 4,     /* a bounded device wait gave up               */
    SAQ_ERR_UNSUPPORTED = 5, /* valid request the build does not support    */
    SAQ_ERR_RANGE = 6        /* an input row is not finite or lies outside
                                the range of the projection's operand format;
                                the outputs of that call are invalid        */
} saq_status;

/* Arithmetic of the projection GEMM (Sec. 5.1 combined matrix).  Quantization
 * and code adjustment always run in FP32.
 *   SAQ_PREC_FP32: FP32 inputs; tensor-core GEMM with a three-term FP16
 *                  split of both operands and FP32 accumulation (error on
 *                  the order of FP32 rounding).
 *   SAQ_PREC_FP32_SIMT: FP32 CUDA-core GEMM (reference-grade, slow).
 *   SAQ_PREC_BF16: BF16 operands on the tensor cores, FP32 accumulation.
 *   SAQ_PREC_FP8:  FP8 e4m3 operands with per-segment scales, FP32
 *                  accumulation. */
typedef enum {
    SAQ_PREC_FP32 = 0,
    SAQ_PREC_BF16 = 1,
    SAQ_PREC_FP8 = 2,
    SAQ_PREC_FP32_SIMT = 3
} saq_precision;

/* Fit parameters (Sec. 4.1-4.2; Sec. 3.1 for rounds). */
typedef struct {
    double avg_bits;          /* bit quota Q_quota = round(avg_bits * d)      */
    int32_t max_bits;         /* valid per-segment bits are 0..max_bits (<=8) */
    int32_t rounds;           /* code-adjustment rounds r of Algorithm 1      */
    int32_t seg_granularity;  /* segment length multiple g (paper: 64)        */
    int32_t precision;        /* saq_precision of the projection GEMM         */
    double tie_frac;          /* plan: fewest segments within (1+tie_frac) of
                                 the least modelled error (paper: 0.1%)      */
    uint64_t seed;            /* seed of the per-segment random rotations     */
} saq_params;

/* One segment of a quantization plan (Sec. 4.1 tuple (Seg, B)): PCA
 * dimensions [start, start+len) quantized with `bits` bits each; bits == 0
 * drops the segment. */
typedef struct {
    int32_t start;
    int32_t len;
    int32_t bits;
} saq_segment;

/* Fill *p with the defaults: avg_bits 4, max_bits 8, rounds 6, granularity
 * 64, precision FP32, tie_frac 1e-3, seed 4. */
void saq_params_init(saq_params *p);

/*
 * Fit a model on n rows of X_dev (device, row-major n x d FP32):
 * mean c and FP64 covariance on the GPU, eigen-decomposition (sigma^2
 * descending, Sec. 4.1), plan by Algorithm 2 with
 * ERROR(Seg,B) = sum sigma_i^2 2^-B (Eq. seg-err, empirical-variance form),
 * a seeded random orthonormal matrix per kept segment, and the combined
 * matrix W = blockdiag(R_s) V_kept^T (Sec. 5.1).  Synchronous: returns after
 * the model is ready.  n >= 2, d >= 1.  *out receives a new model owned by
 * the caller (free with saq_model_free).
 */
saq_status saq_fit(const float *X_dev, int64_t n, int32_t d,
                   const saq_params *p, saq_model **out, void *stream);

/*
 * Build a model from explicit host arrays (FP64): mean[d]; plan[nseg]
 * covering [0, d) in order; W[d_kept x d] row-major, the rows of the kept
 * segments in plan order (d_kept = sum of len over segments with bits > 0);
 * sig2[d] optional (may be NULL).  Only p->rounds and p->precision are used.
 * Copies everything; synchronous.
 */
saq_status saq_model_create(int32_t d, const double *mean, const double *W,
                            const saq_segment *plan, int32_t nseg,
                            const double *sig2, const saq_params *p,
                            saq_model **out);

void saq_model_free(saq_model *m);

/* Model queries.  Code layout: per vector, code_bytes bytes; per kept
 * segment in plan order, `bits` bit-planes, most significant first; plane p
 * holds bit (bits-1-p) of every code of the segment as ceil(len/64)
 * little-endian 64-bit words (coordinate i -> word i/64, bit i%64).  The
 * first b planes of a segment are its b-bit prefix code (Sec. 3.2).
 * Factor layout: per vector factor_count FP32 values:
 * [ |o_r - c|^2, then per kept segment |o_s|, cos_s ], where cos_s is the
 * cosine between the adjusted quantized vector and o_s (Sec. 3.1 end). */
size_t saq_code_bytes(const saq_model *m);
int32_t saq_factor_count(const saq_model *m);
int32_t saq_model_dim(const saq_model *m);
int32_t saq_model_kept_dim(const saq_model *m);
int32_t saq_model_num_segments(const saq_model *m);   /* all, incl. dropped */
saq_status saq_model_get_plan(const saq_model *m, saq_segment *out, int32_t cap);
saq_status saq_model_get_mean(const saq_model *m, double *out /* d */);
saq_status saq_model_get_matrix(const saq_model *m, double *out /* d_kept x d */);
saq_status saq_model_get_variances(const saq_model *m, double *out /* d */);
/* Change the GEMM precision (saq_precision) or the number of adjustment
 * rounds of an existing model.  Synchronous; not concurrent with encodes. */
saq_status saq_model_set_precision(saq_model *m, int32_t precision);
saq_status saq_model_set_rounds(saq_model *m, int32_t rounds);

/*
 * Encode n vectors (the hot path).  X_dev: device, row-major n x d FP32.
 * Per vector: o = W (x - c) (Sec. 3.1 Eq. rotate with the combined PCA +
 * segment-rotation matrix of Sec. 5.1); per kept segment: v_max, Delta and
 * the initial code of Eq. find_nearest_code (o = v_max clamps to 2^B - 1),
 * then r rounds of Algorithm 1 (+Delta tried before -Delta, a move kept only
 * if it stays in range and strictly raises cos(x, o); a round without a move
 * ends the segment early, which changes no result); then the factors and the
 * bit-plane codes.  Outputs: codes_dev n x code_bytes, factors_dev
 * n x factor_count FP32.  Asynchronous on `stream`.  n == 0 is a no-op.
 * Rows are processed in chunks of about 1 GB of projected rows (projection,
 * then quantization, per chunk).  Scratch memory (5 bytes per row and kept
 * dimension of a chunk, plus 4 per row and kept segment) comes from a
 * stream-ordered pool the library keeps per device (memory up to 8 GB stays
 * cached between calls) and is returned before the call's work completes on
 * the stream.
 */
saq_status saq_encode(const saq_model *m, const float *X_dev, int64_t n,
                      uint8_t *codes_dev, float *factors_dev, void *stream);

/*
 * Same as saq_encode, with host buffers: the rows are copied to the device
 * in chunks of about 128 MB, encoded and the codes and factors copied back,
 * through three staging slots, with the copy-in of the next chunk and the
 * copy-out of the previous one (on two streams of their own) overlapping the
 * encode of the current one.  Page-locked host memory is strongly
 * recommended.  Synchronous: returns when the outputs are in host memory.
 */
saq_status saq_encode_host(const saq_model *m, const float *X_host, int64_t n,
                           uint8_t *codes_host, float *factors_host,
                           void *stream);

/*
 * The two halves of saq_encode, for testing and for callers that already
 * hold projected vectors.
 * saq_project: O_dev (n x d_kept FP32, row-major) = W (x - c) with the
 *   model's precision, norms2_dev[n] = |x - c|^2.
 * saq_quantize_projected: quantize and adjust O_dev as saq_encode does and
 *   write codes and factors; factor 0 of each vector is taken from
 *   norms2_dev.
 */
saq_status saq_project(const saq_model *m, const float *X_dev, int64_t n,
                       float *O_dev, float *norms2_dev, void *stream);
saq_status saq_quantize_projected(const saq_model *m, const float *O_dev,
                                  const float *norms2_dev, int64_t n,
                                  uint8_t *codes_dev, float *factors_dev,
                                  void *stream);
/* The same with a layout flag: interleaved != 0 selects the layout the
 * encode uses internally, rows in groups of 32:
 *   O_dev[((i / 32) * d_kept + j) * 32 + i % 32] = o_i[j],
 * with room for ceil(n / 32) * 32 rows.  interleaved == 0 is the row-major
 * layout of saq_project / saq_quantize_projected. */
saq_status saq_project_ex(const saq_model *m, const float *X_dev, int64_t n,
                          float *O_dev, float *norms2_dev, int32_t interleaved,
                          void *stream);
saq_status saq_quantize_projected_ex(const saq_model *m, const float *O_dev,
                                     const float *norms2_dev, int64_t n,
                                     uint8_t *codes_dev, float *factors_dev,
                                     int32_t interleaved, void *stream);

/*
 * saq_encode for callers that cannot allocate device memory.  The paper has
 * no counterpart; this is a deployment variant of the encode above.
 *
 * Some callers may not call cudaMalloc (or any allocating routine) at encode
 * time: a framework that owns all device memory through its own allocator,
 * so a driver-level allocation would fail or fragment its pool; an ingest
 * thread with a hard latency budget, where an allocation can block and
 * synchronise the device; or a host (a database extension, a plugin) that
 * forbids driver allocations from inside its callbacks.  This entry point
 * allocates nothing: its scratch (the projected rows, 4 bytes per row and kept
 * dimension, their codes during adjustment, 1 byte, and the largest
 * magnitude per row and kept segment, 4 bytes) lives in a fixed 32 MiB array
 * in the library's device memory, which every GPU that loads the library
 * keeps until the process exits.
 *
 * Limit: ceil(n / 32) * 32 * (5 * d_kept + 4 * segments) bytes <= 32 MiB,
 * e.g. 6,944 rows at d_kept = 960 in 4 kept segments; larger n is rejected
 * with SAQ_ERR_INVALID before any launch (the message states the largest n
 * for the model).  Arguments and outputs
 * are as for saq_encode.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  The looked-up address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys and
 * recreates the device's primary context) the kept address is stale, so
 * this entry point must not be used on that device again.  Every call shares the one array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  The array keeps the last call's contents:
 * each call clears the per-segment maxima (which must start at zero) on its
 * stream before using them; the rest is written before it is read.
 */
saq_status saq_encode_noalloc(const saq_model *m, const float *X_dev, int64_t n,
                              uint8_t *codes_dev, float *factors_dev, void *stream);

/*
 * Estimated squared distances dist_dev[q * n + v] between query q (rows of
 * Q_dev, device nq x d FP32) and encoded vector v:
 *   |o_r - q_r|^2 ~ |o_r - c|^2 + |q_r - c|^2 - 2 sum_s est_s      (Eq. 3)
 *   est_s = |o_s| <u_s, q_s> / (|u_s| cos_s),  u_s = 2 c_a - (2^B - 1)
 * which is the estimator <o_bar_a, q>/<o_bar_a, o> |o|^2 of Sec. 3.2 per
 * segment, with q_s the query rotated by the same matrix.  prefix_bits > 0
 * uses the b = min(prefix_bits, B) most significant bits of every code
 * (progressive approximation, Sec. 3.2) with the stored factors; 0 uses all
 * bits.  Asynchronous on `stream`.
 */
saq_status saq_estimate_dist(const saq_model *m, const uint8_t *codes_dev,
                             const float *factors_dev, int64_t n,
                             const float *Q_dev, int64_t nq,
                             int32_t prefix_bits, float *dist_dev,
                             void *stream);

/*
 * Serialise a model (mean, plan, W, sigma^2, rounds, precision and, when
 * the model carries one, the PCA basis of saq_model_set_basis) into a
 * versioned little-endian blob (version 2; import also reads version 1,
 * which has no basis).  With buf == NULL, *len receives the size.
 * Otherwise *len is the capacity of buf and receives the bytes written.
 */
saq_status saq_model_export(const saq_model *m, void *buf, size_t *len);
saq_status saq_model_import(const void *buf, size_t len, saq_model **out);

/*
 * Quantization plan search alone (Sec. 4.2 Algorithm 2), host only, no GPU:
 * sig2[d] the per-dimension variances sorted descending, g the segment
 * granularity, quota_bits the bit quota, max_bits <= 8, tie_frac the
 * "fewest segments within (1 + tie_frac) of the least error" rule.  Writes
 * up to cap segments to out, their number to *nseg and the plan's modelled
 * error to *err (may be NULL).  Same plan as saq_fit computes.
 */
saq_status saq_plan_search(const double *sig2, int32_t d, int32_t g, int64_t quota_bits,
                           int32_t max_bits, double tie_frac, saq_segment *out, int32_t cap,
                           int32_t *nseg, double *err);

/* 1 if the model's projection runs on the tensor cores (tcgen05), 0 if on
 * the CUDA cores (SAQ_PREC_FP32_SIMT, or d not a multiple of 4). */
int32_t saq_model_uses_tensor_cores(const saq_model *m);

/* Synchronise `stream`, then report whether a bounded device wait inside the
 * model's kernels gave up (SAQ_ERR_TIMEOUT) or an input row was out of range
 * (SAQ_ERR_RANGE) since the last check; the flag is cleared.  Failure
 * detection for the asynchronous entry points (saq_encode_host, which is
 * synchronous, reports both itself).  The range check of the tensor-core
 * projection is on the scaled, centred squared row norm |(x - c) s|^2, s the
 * power of two that maps the fitted per-coordinate rms to 8 (FP32 split):
 * it fires at 65504^2, the square of FP16's largest value, i.e. when a row's
 * |x - c| reaches about 8,000 times the fitted rms (a coordinate could
 * overflow the split there); the BF16 and FP8 forms flag non-finite rows
 * only (E4M3 saturates at 448, see SAQ_PREC_FP8). */
saq_status saq_check_device(const saq_model *m, void *stream);

/* Failure detection (no counterpart in the paper): the bound, in
 * nanoseconds, of every pipeline wait inside the tensor-core projection
 * (TMA producer, MMA issuer and converters waiting on one another) for
 * launches that start after the call; 0 restores the default of 2 s.  A
 * wait that reaches its bound raises the device error flag, every role
 * leaves its loop, the copies and MMAs already in flight are drained (those
 * drain waits keep the 2 s bound), tensor memory is freed and the kernel
 * returns; the next saq_check_device (or saq_encode_host itself) returns
 * SAQ_ERR_TIMEOUT and clears the flag.  Process-wide; meant for tests of
 * that path (a bound of a few nanoseconds makes the waits run out) and for
 * hosts that want a tighter watchdog.  Always SAQ_OK. */
saq_status saq_set_wait_limit(uint64_t ns);

/* ------------------------------------------------------------------------
 * Serving: continuous-batching ingest over several resident collections.
 * (The paper's encoder is offline; this runtime applies the encode of
 * saq_encode to a stream of insert requests.)
 *
 * Each collection is a fitted model kept resident on the device.  Requests
 * (host rows of one collection) queue on submit; a scheduler thread forms
 * batches as slots free up: a batch takes the queued requests oldest first,
 * from up to 4 collections whose models use the same tensor-core precision,
 * at most max_batch_rows rows in all (large requests are split across
 * batches), and encodes them with ONE persistent projection launch and ONE
 * persistent quantize/adjust/pack launch over all its collections (one CTA
 * per SM, resp. as many blocks as stay resident, taking the batch's tiles and
 * items from device work counters), on one of `slots` streams, between one
 * copy-in and one copy-out per request piece.  A model
 * on the CUDA-core projection gets batches of its own.  Requests that arrive
 * while others are on the GPU join the next batch, so the copies and kernels
 * of different batches overlap.
 * Admission is by HBM budget: a batch's device memory (inputs, codes,
 * factors and projection scratch: 4 d + code_bytes + 4 factor_count bytes per
 * row plus the encode's scratch) is taken from the library's stream-ordered
 * pool when the batch is formed and returned when it completes, and a batch
 * is formed only with the pieces of requests that fit in hbm_budget_bytes
 * beside the batches already in flight (a request that does not fit waits,
 * whole or in part, for earlier batches to complete; each time the budget
 * holds back queued work counts as a deferred batch).  Open fails with
 * SAQ_ERR_OOM if one batch of max_batch_rows rows of some collection alone
 * exceeds the budget.  Results are identical to saq_encode on the same rows:
 * every row is encoded independently.  A bounded wait of a batch's
 * projection that gave up (SAQ_ERR_TIMEOUT) or an input row out of range
 * (SAQ_ERR_RANGE) fails every request with rows in that batch.
 * ------------------------------------------------------------------------ */
typedef struct saq_ingest saq_ingest;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory the batches in flight may hold */
    int32_t max_batch_rows;   /* rows per batch (>= 1), over all its collections */
    int32_t slots;            /* concurrent batches (streams), 1..64          */
} saq_ingest_params;

typedef struct {
    uint64_t submitted, completed, rows_completed, batches;
    double p50_latency_s, p99_latency_s, max_latency_s;  /* submit -> done */
    double busy_s;            /* wall time between first submit and last completion */
    uint64_t mixed_batches;   /* batches that held rows of several collections */
    uint64_t deferred_batches;/* times queued work waited for budget          */
    size_t peak_bytes_in_flight; /* most device memory the batches held at once */
} saq_ingest_stats;

/* models[n_models] stay owned by the caller and must outlive the service. */
saq_status saq_ingest_open(saq_model *const *models, int32_t n_models,
                           const saq_ingest_params *p, saq_ingest **out);
/* Queue n rows (host, row-major n x d of the collection's model) whose codes
 * and factors go to codes_host / factors_host (sized as for saq_encode).
 * Page-locked host memory is recommended.  Buffers must stay valid until the
 * request completes.  Never blocks on the GPU; *ticket identifies it. */
saq_status saq_ingest_submit(saq_ingest *s, int32_t collection, const float *X_host,
                             int64_t n, uint8_t *codes_host, float *factors_host,
                             uint64_t *ticket);
/* *done = 1 once the request's outputs are in host memory. */
saq_status saq_ingest_poll(saq_ingest *s, uint64_t ticket, int32_t *done);
/* Wait up to timeout_ms (< 0: no limit) for the request; SAQ_ERR_TIMEOUT if
 * it is still in flight.  *latency_s (may be NULL) receives submit-to-done. */
saq_status saq_ingest_wait(saq_ingest *s, uint64_t ticket, int32_t timeout_ms,
                           double *latency_s);
saq_status saq_ingest_get_stats(saq_ingest *s, saq_ingest_stats *out);
/* Waits for all queued and in-flight requests, then frees the service. */
saq_status saq_ingest_close(saq_ingest *s);

/* Number of CUDA kernels the library has launched in this process so far
 * (all threads, all devices).  Diagnostic; never reset. */
uint64_t saq_kernel_launch_count(void);

/* Multi-stage distance estimation (Sec. 4.3).  The kept segments are taken
 * in plan order, i.e. by decreasing PCA variance.  After t stages the first
 * t segments contribute their estimates est_s (as in saq_estimate_dist) and
 * every remaining one its Chebyshev bound m * sigma_Seg(q), where
 *   sigma_Seg(q)^2 = sum_{i in Seg} sigma_i^2 (v_i . (q_r - c))^2
 * is the variance of <o_seg, q_seg> over the data (v_i, sigma_i^2: PCA
 * direction and variance of dimension i), so |<o_seg, q_seg>| < m sigma_Seg
 * with probability >= 1 - 1/m^2:
 *   bounds[(q*n + v)*(k+1) + t] = |o_r - c|^2 + |q_r - c|^2
 *                                 - 2 (sum_{s<t} est_s + m sum_{s>=t} sigma_s(q)),
 * t = 0 .. k (k = kept segments).  t = k equals saq_estimate_dist; dropped
 * segments contribute nothing, as there.  A search prunes vector v for
 * query q as soon as a stage's bound exceeds its current best distance.
 * codes_dev/factors_dev: n rows as written by saq_encode; Q_dev: nq x d
 * FP32 row-major; bounds_dev: nq x n x (k+1) FP32, caller-owned.  m_conf
 * (the paper's m) must be finite and >= 0.  The model must carry the PCA
 * basis: saq_fit records it; a model built by saq_model_create needs
 * saq_model_set_basis, else SAQ_ERR_UNSUPPORTED.  Asynchronous on `stream`. */
saq_status saq_estimate_staged(const saq_model *m, const uint8_t *codes_dev,
                               const float *factors_dev, int64_t n, const float *Q_dev, int64_t nq,
                               float m_conf, float *bounds_dev, void *stream);

/* The PCA directions of the kept dimensions (Sec. 4.1), for the bounds of
 * saq_estimate_staged: Vt is d_kept x d row-major FP64, row r = v_i^T for
 * the r-th kept dimension in plan order (i = start of its segment + offset),
 * i.e. W = blockdiag(R_s) Vt.  Copied; exported with the model.
 * SAQ_ERR_INVALID on NULL or non-finite input.  saq_model_has_basis
 * returns 1 if the model carries one. */
saq_status saq_model_set_basis(saq_model *m, const double *Vt);
int32_t saq_model_has_basis(const saq_model *m);

/* Instruction ceiling of the code adjustment (diagnostic; no counterpart in
 * the paper).  Runs the adjustment's own per-coordinate step (Algorithm 1 in
 * the closed form of saq_encode) on coordinates held in registers, with no
 * memory traffic, at warps_per_sm resident warps per SM (4, 8, ..., 64;
 * the quantize kernel runs at 32) and B = bits, on the current device and
 * the legacy default stream, and writes the lane-steps per second
 * (coordinate trials of one vector-segment each) to *lane_steps_per_s.
 * Synchronous.  The quantize kernel's own rate of lane-steps measured
 * against it shows how much of the step's issue ceiling it reaches.
 * SAQ_ERR_INVALID on bad arguments. */
saq_status saq_quantize_step_ceiling(int32_t warps_per_sm, int32_t bits,
                                     double *lane_steps_per_s);

/* Kernel timing (diagnostic; no counterpart in the paper).  While enabled,
 * every kernel the library launches is bracketed by two CUDA events recorded
 * on its own stream, just before the launch and just after it, so that each
 * interval is that launch's device time even when streams overlap.
 * saq_kernel_timing(1) clears the record and starts recording (all threads,
 * all devices); saq_kernel_timing(0) stops and keeps the record.  saq_kernel_times() waits for the
 * recorded events and writes, for kind k < kinds, the summed milliseconds
 * ms[k] and the number of launches launches[k]:
 *   k = 0  projection (tensor-core or CUDA-core GEMM of the encode),
 *   k = 1  quantize / adjust / pack (Eq. find_nearest_code, Algorithm 1),
 *   k = 2  everything else (v_max pass, layout changes, estimator, fit).
 * kinds must be 1..3; ms and launches are host arrays of `kinds` entries.
 * SAQ_ERR_INVALID on bad arguments, SAQ_ERR_CUDA if an event failed. */
saq_status saq_kernel_timing(int enable);
saq_status saq_kernel_times(double *ms, int64_t *launches, int kinds);

/* Message of the calling thread's last failed call ("" if none). */
const char *saq_last_error(void);
const char *saq_status_string(saq_status s);

#ifdef __cplusplus
}
#endif

#endif /* SAQ_H */
