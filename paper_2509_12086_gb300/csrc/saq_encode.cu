// saq_encode.cu -- C-ABI entry points of the encode hot path and of the
// estimator: argument checks, scratch management and kernel sequencing.
#include <algorithm>
#include <cmath>

#include "saq_internal.h"

namespace saq {

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

saq_status check_device(const saq_model *m) {
    int dev = -1;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev != m->device)
        return set_error(SAQ_ERR_INVALID, "model lives on device %d, current device is %d",
                         m->device, dev);
    return SAQ_OK;
}

// Rows per chunk so that the projected chunk stays within `budget` bytes.
int64_t chunk_rows(const saq_model *m, int64_t n, size_t budget) {
    const int64_t per = std::max<int64_t>(1, (int64_t)m->dk * 4);
    int64_t r = (int64_t)(budget / (size_t)per);
    r = std::max<int64_t>(r, 256);
    r = (r / 128) * 128;
    return std::min<int64_t>(r, n);
}

}  // namespace

bool use_tc(const saq_model *m) {
    return m->precision != SAQ_PREC_FP32_SIMT && m->tc.precision == m->precision &&
           tc_supported(m);
}

namespace {
// Scratch of an encode of up to `rows` rows: interleaved projected rows (FP32),
// their codes during adjustment (bytes), and v_max per row and kept segment.
struct ScratchParts {
    float *Oi;
    uint8_t *cs;
    float *vmax;
    size_t vmax_bytes;
};
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
ScratchParts scratch_parts(const saq_model *m, void *scratch, int64_t rows) {
    const size_t r32 = (size_t)((rows + 31) / 32 * 32);
    const size_t elems = r32 * (size_t)std::max(1, m->dk);
    uint8_t *b = static_cast<uint8_t *>(scratch);
    ScratchParts p;
    p.Oi = reinterpret_cast<float *>(b);
    p.cs = b + align256(elems * sizeof(float));
    p.vmax = reinterpret_cast<float *>(p.cs + align256(elems));
    p.vmax_bytes = r32 * std::max<size_t>(1, m->kept.size()) * sizeof(float);
    return p;
}
}  // namespace

size_t encode_scratch_bytes(const saq_model *m, int64_t rows) {
    const size_t r32 = (size_t)((rows + 31) / 32 * 32);
    const size_t elems = r32 * (size_t)std::max(1, m->dk);
    return align256(elems * sizeof(float)) + align256(elems) +
           align256(r32 * std::max<size_t>(1, m->kept.size()) * sizeof(float));
}

// Projection of rows [0, n) into O and |x - c|^2 into norms (stride); with
// the interleaved layout and vmax != NULL also v_max per row and segment.
saq_status project_rows(const saq_model *m, const float *X, int64_t n, float *O, int64_t ldo,
                        int layout, float *norms, int64_t nstride, float *vmax, cudaStream_t s,
                        int *err) {
    if (use_tc(m)) {
        if (vmax && layout == kInterleaved)
            SAQ_CUDA_CHECK(cudaMemsetAsync(vmax, 0, sizeof(float) * (size_t)((n + 31) / 32 * 32) *
                                                       m->kept.size(), s));
        return launch_project_tc(m, X, n, O, ldo, layout, norms, nstride, vmax, err, s);
    }
    saq_status st = launch_project_simt(m, X, n, O, ldo, layout, s);
    if (st != SAQ_OK) return st;
    st = launch_rownorm2(m, X, n, norms, nstride, s);
    if (st != SAQ_OK) return st;
    if (vmax && layout == kInterleaved) st = launch_seg_vmax(m, O, n, vmax, s);
    return st;
}

// Quantize rows [0, n) whose interleaved projection (and v_max) sit in
// `scratch` (sized by encode_scratch_bytes for rows_cap rows).
saq_status quantize_rows(const saq_model *m, void *scratch, int64_t rows_cap, int64_t n,
                         uint8_t *codes, float *factors, cudaStream_t s) {
    const ScratchParts p = scratch_parts(m, scratch, rows_cap);
    return launch_caq1(m, p.Oi, n, p.cs, p.vmax, codes, factors, s);
}

// The whole encode of rows [0, n) on stream s with a scratch for `rows` rows.
saq_status encode_rows(const saq_model *m, const float *X, int64_t n, uint8_t *codes,
                       float *factors, void *scratch, int64_t rows, cudaStream_t s, int *err) {
    for (int64_t r0 = 0; r0 < n; r0 += rows) {
        const int64_t nr = std::min(rows, n - r0);
        const ScratchParts p = scratch_parts(m, scratch, rows);
        saq_status st = project_rows(m, X + r0 * m->d, nr, p.Oi, m->dk, kInterleaved,
                                     factors + r0 * m->nf, m->nf, p.vmax, s, err);
        if (st != SAQ_OK) return st;
        st = quantize_rows(m, scratch, rows, nr, codes + r0 * (int64_t)m->code_bytes,
                           factors + r0 * m->nf, s);
        if (st != SAQ_OK) return st;
    }
    return SAQ_OK;
}

// Rows of up to kMaxGroups models in one persistent projection launch and one
// persistent quantize launch (a serving batch of several collections); see
// saq_internal.h.
saq_status encode_grouped(const EncodeJob *jobs, int njobs, cudaStream_t s, int *err, int *queue) {
    if (njobs < 1 || njobs > kMaxGroups)
        return set_error(SAQ_ERR_INVALID, "1..%d models per grouped encode", kMaxGroups);
    ProjJob pj[kMaxGroups];
    CaqJob cj[kMaxGroups];
    int np = 0;
    for (int i = 0; i < njobs; ++i) {
        const EncodeJob &j = jobs[i];
        if (j.n <= 0) continue;
        if (j.m->dk == 0) {
            saq_status st = launch_rownorm2(j.m, j.X, j.n, j.factors, j.m->nf, s);
            if (st != SAQ_OK) return st;
            continue;
        }
        if (!use_tc(j.m))
            return set_error(SAQ_ERR_INVALID, "grouped encode needs tensor-core models");
        const ScratchParts p = scratch_parts(j.m, j.scratch, j.n);
        SAQ_CUDA_CHECK(cudaMemsetAsync(p.vmax, 0, p.vmax_bytes, s));
        pj[np] = ProjJob{j.m, j.X, j.n, p.Oi, j.factors, j.m->nf, p.vmax, err};
        cj[np] = CaqJob{j.m, p.Oi, j.n, p.cs, p.vmax, j.codes, j.factors};
        ++np;
    }
    if (np == 0) return SAQ_OK;
    SAQ_CUDA_CHECK(cudaMemsetAsync(queue, 0, 2 * sizeof(int), s));
    saq_status st = launch_project_tc_grouped(pj, np, queue, s);
    if (st != SAQ_OK) return st;
    return launch_caq1_grouped(cj, np, queue + 1, s);
}

}  // namespace saq

using namespace saq;

extern "C" {

saq_status saq_encode(const saq_model *m, const float *X_dev, int64_t n, uint8_t *codes_dev,
                      float *factors_dev, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!X_dev || !factors_dev || (m->code_bytes > 0 && !codes_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(X_dev) || !aligned16(codes_dev) || !aligned16(factors_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (m->dk == 0) return launch_rownorm2(m, X_dev, n, factors_dev, m->nf, s);
    // chunks of about 1 GB of projected rows, each projected then quantized
    // on `s` (measured at d = 960: 1 GB chunks run as fast as smaller chunks
    // whose projection overlaps the previous chunk's quantization on a
    // second stream, and need half the scratch)
    const int64_t rows = chunk_rows(m, n, (size_t)1024 << 20);
    const size_t sb = encode_scratch_bytes(m, rows);
    void *scratch = nullptr;
    cudaError_t e = scratch_alloc(&scratch, sb, s);
    if (e != cudaSuccess)
        return set_error(SAQ_ERR_OOM, "scratch allocation failed: %s", cudaGetErrorString(e));
    st = encode_rows(m, X_dev, n, codes_dev, factors_dev, scratch, rows, s);
    cudaFreeAsync(scratch, s);
    return st;
}

saq_status saq_project(const saq_model *m, const float *X_dev, int64_t n, float *O_dev,
                       float *norms2_dev, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!X_dev || !norms2_dev || (m->dk > 0 && !O_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(X_dev) || !aligned16(O_dev) || !aligned16(norms2_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    return project_rows(m, X_dev, n, O_dev, m->dk, kRowMajor, norms2_dev, 1, nullptr,
                        (cudaStream_t)stream);
}

saq_status saq_project_ex(const saq_model *m, const float *X_dev, int64_t n, float *O_dev,
                          float *norms2_dev, int32_t interleaved, void *stream) {
    clear_error();
    if (!interleaved) return saq_project(m, X_dev, n, O_dev, norms2_dev, stream);
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!X_dev || !norms2_dev || (m->dk > 0 && !O_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(X_dev) || !aligned16(O_dev) || !aligned16(norms2_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    return project_rows(m, X_dev, n, O_dev, m->dk, kInterleaved, norms2_dev, 1, nullptr,
                        (cudaStream_t)stream);
}

saq_status saq_quantize_projected_ex(const saq_model *m, const float *O_dev,
                                     const float *norms2_dev, int64_t n, uint8_t *codes_dev,
                                     float *factors_dev, int32_t interleaved, void *stream) {
    clear_error();
    if (!interleaved)
        return saq_quantize_projected(m, O_dev, norms2_dev, n, codes_dev, factors_dev, stream);
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!norms2_dev || !factors_dev || (m->dk > 0 && (!O_dev || !codes_dev)))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(O_dev) || !aligned16(codes_dev) || !aligned16(factors_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = launch_copy_strided(norms2_dev, 1, factors_dev, m->nf, n, s);
    if (st != SAQ_OK || m->dk == 0) return st;
    void *scratch = nullptr;
    if (scratch_alloc(&scratch, encode_scratch_bytes(m, n), s) != cudaSuccess)
        return set_error(SAQ_ERR_OOM, "scratch allocation failed");
    const ScratchParts p = scratch_parts(m, scratch, n);
    st = launch_seg_vmax(m, O_dev, n, p.vmax, s);
    if (st == SAQ_OK) st = launch_caq1(m, O_dev, n, p.cs, p.vmax, codes_dev, factors_dev, s);
    cudaFreeAsync(scratch, s);
    return st;
}

saq_status saq_quantize_projected(const saq_model *m, const float *O_dev,
                                  const float *norms2_dev, int64_t n, uint8_t *codes_dev,
                                  float *factors_dev, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!norms2_dev || !factors_dev || (m->dk > 0 && (!O_dev || !codes_dev)))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(O_dev) || !aligned16(codes_dev) || !aligned16(factors_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = launch_copy_strided(norms2_dev, 1, factors_dev, m->nf, n, s);
    if (st != SAQ_OK || m->dk == 0) return st;
    void *scratch = nullptr;
    cudaError_t e = scratch_alloc(&scratch, encode_scratch_bytes(m, n), s);
    if (e != cudaSuccess)
        return set_error(SAQ_ERR_OOM, "scratch allocation failed: %s", cudaGetErrorString(e));
    const ScratchParts p = scratch_parts(m, scratch, n);
    st = launch_interleave(O_dev, m->dk, n, m->dk, p.Oi, s);
    if (st == SAQ_OK) st = launch_seg_vmax(m, p.Oi, n, p.vmax, s);
    if (st == SAQ_OK) st = quantize_rows(m, scratch, n, n, codes_dev, factors_dev, s);
    cudaFreeAsync(scratch, s);
    return st;
}

saq_status saq_encode_host(const saq_model *m, const float *X_host, int64_t n,
                           uint8_t *codes_host, float *factors_host, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0) return set_error(SAQ_ERR_INVALID, "n < 0");
    if (n == 0) return SAQ_OK;
    if (!X_host || !factors_host || (m->code_bytes > 0 && !codes_host))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // kSlots staging slots of about 128 MB of rows; a copy-in stream and a
    // copy-out stream (the two copy engines) run beside the encode on `s`:
    // the copy-in of chunk i+1 and the copy-out of chunk i-1 overlap the
    // encode of chunk i.  The call is bound by the copy-in, so chunks are
    // kept small enough that the last chunk's encode and copy-out, which
    // follow the last copy-in, are short (512 MB chunks: 20.7 ms per 1M rows
    // of d = 960, 128 MB: 19.8 ms, 64 MB: 20.3 ms).  Buffers come from the
    // stream-ordered pool.
    constexpr int kSlots = 3;
    const int64_t rows = std::min<int64_t>(
        n, std::max<int64_t>(32, ((int64_t)(128 << 20) / (4 * (int64_t)m->d)) / 32 * 32));
    auto round16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t xb = round16(sizeof(float) * (size_t)rows * m->d);
    const size_t cb = round16(m->code_bytes * (size_t)rows);
    const size_t fb = round16(sizeof(float) * (size_t)rows * m->nf);
    const size_t slot = xb + cb + fb;
    const size_t ob = m->dk > 0 ? encode_scratch_bytes(m, rows) : 0;
    uint8_t *buf = nullptr;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ready = nullptr, done_in = nullptr, done_out = nullptr;
    cudaEvent_t in_done[kSlots] = {}, enc_done[kSlots] = {}, out_done[kSlots] = {};
    auto cleanup = [&]() {
        // join the copy streams into `s`, then return the buffers
        if (d2h && done_out) {
            cudaEventRecord(done_out, d2h);
            cudaStreamWaitEvent(s, done_out, 0);
        }
        if (h2d && done_in) {
            cudaEventRecord(done_in, h2d);
            cudaStreamWaitEvent(s, done_in, 0);
        }
        if (buf) cudaFreeAsync(buf, s);
        cudaStreamSynchronize(s);
        if (h2d) cudaStreamDestroy(h2d);
        if (d2h) cudaStreamDestroy(d2h);
        for (cudaEvent_t e : {ready, done_in, done_out}) if (e) cudaEventDestroy(e);
        for (int i = 0; i < kSlots; ++i)
            for (cudaEvent_t e : {in_done[i], enc_done[i], out_done[i]}) if (e) cudaEventDestroy(e);
    };
    bool ok = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t *e : {&ready, &done_in, &done_out})
        ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < kSlots && ok; ++i)
        for (cudaEvent_t *e : {&in_done[i], &enc_done[i], &out_done[i]})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cleanup();
        return set_error(SAQ_ERR_CUDA, "stream/event creation failed");
    }
    if (scratch_alloc((void **)&buf, slot * kSlots + ob, s) != cudaSuccess) {
        buf = nullptr;
        cleanup();
        return set_error(SAQ_ERR_OOM, "staging allocation failed");
    }
    void *O = buf + slot * kSlots;
    // the copy streams may use the buffers once the allocation is ordered
    cudaEventRecord(ready, s);
    cudaStreamWaitEvent(h2d, ready, 0);
    cudaStreamWaitEvent(d2h, ready, 0);
    int64_t chunk = 0;
    for (int64_t r0 = 0; r0 < n && st == SAQ_OK; r0 += rows, ++chunk) {
        const int sl = (int)(chunk % kSlots);
        const int64_t nr = std::min(rows, n - r0);
        uint8_t *base = buf + slot * (size_t)sl;
        float *dx = (float *)base;
        uint8_t *dc = base + xb;
        float *df = (float *)(base + xb + cb);
        // the slot's previous copy-out must be done before it is refilled
        if (chunk >= kSlots) cudaStreamWaitEvent(h2d, out_done[sl], 0);
        cudaMemcpyAsync(dx, X_host + r0 * m->d, sizeof(float) * (size_t)nr * m->d,
                        cudaMemcpyHostToDevice, h2d);
        cudaEventRecord(in_done[sl], h2d);
        cudaStreamWaitEvent(s, in_done[sl], 0);
        if (m->dk == 0) st = launch_rownorm2(m, dx, nr, df, m->nf, s);
        else st = encode_rows(m, dx, nr, dc, df, O, rows, s);
        cudaEventRecord(enc_done[sl], s);
        cudaStreamWaitEvent(d2h, enc_done[sl], 0);
        if (m->code_bytes)
            cudaMemcpyAsync(codes_host + r0 * (int64_t)m->code_bytes, dc, m->code_bytes * (size_t)nr,
                            cudaMemcpyDeviceToHost, d2h);
        cudaMemcpyAsync(factors_host + r0 * m->nf, df, sizeof(float) * (size_t)nr * m->nf,
                        cudaMemcpyDeviceToHost, d2h);
        cudaEventRecord(out_done[sl], d2h);
    }
    cleanup();
    cudaError_t e = cudaGetLastError();
    if (st != SAQ_OK) return st;
    if (e != cudaSuccess) return set_error(SAQ_ERR_CUDA, "encode_host: %s", cudaGetErrorString(e));
    // the call is synchronous: a bounded wait that gave up or an input row
    // out of range is reported here, not left for saq_check_device
    if (use_tc(m)) return tc_check_error(m, s);
    return SAQ_OK;
}

int32_t saq_model_uses_tensor_cores(const saq_model *m) { return (m && use_tc(m)) ? 1 : 0; }

saq_status saq_check_device(const saq_model *m, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    SAQ_CUDA_CHECK(cudaStreamSynchronize(s));
    SAQ_CUDA_CHECK(cudaGetLastError());
    return tc_check_error(m, s);
}

saq_status saq_estimate_dist(const saq_model *m, const uint8_t *codes_dev,
                             const float *factors_dev, int64_t n, const float *Q_dev, int64_t nq,
                             int32_t prefix_bits, float *dist_dev, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0 || nq < 0 || prefix_bits < 0) return set_error(SAQ_ERR_INVALID, "negative size");
    if (n == 0 || nq == 0) return SAQ_OK;
    if (!factors_dev || !Q_dev || !dist_dev || (m->code_bytes > 0 && !codes_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(codes_dev) || !aligned16(factors_dev) || !aligned16(Q_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nk = m->kept.size();
    float *qrot = nullptr, *qn2 = nullptr, *vs = nullptr;
    const size_t bq = sizeof(float) * (size_t)nq * std::max(1, m->dk);
    const size_t bv = sizeof(float) * (size_t)n * std::max<size_t>(1, nk);
    if (scratch_alloc((void **)&qrot, bq, s) != cudaSuccess ||
        scratch_alloc((void **)&qn2, sizeof(float) * (size_t)nq, s) != cudaSuccess ||
        scratch_alloc((void **)&vs, bv, s) != cudaSuccess) {
        if (qrot) cudaFreeAsync(qrot, s);
        if (qn2) cudaFreeAsync(qn2, s);
        return set_error(SAQ_ERR_OOM, "scratch allocation failed");
    }
    // queries are rotated with the FP32 CUDA-core projection
    st = launch_project_simt(m, Q_dev, nq, qrot, m->dk, kRowMajor, s);
    if (st == SAQ_OK) st = launch_rownorm2(m, Q_dev, nq, qn2, 1, s);
    if (st == SAQ_OK)
        st = launch_estimate(m, codes_dev, factors_dev, n, qrot, qn2, nq, prefix_bits, vs,
                             dist_dev, s);
    cudaFreeAsync(qrot, s);
    cudaFreeAsync(qn2, s);
    cudaFreeAsync(vs, s);
    return st;
}

saq_status saq_quantize_step_ceiling(int32_t warps_per_sm, int32_t bits,
                                     double *lane_steps_per_s) {
    clear_error();
    if (!lane_steps_per_s) return set_error(SAQ_ERR_INVALID, "NULL output");
    if (warps_per_sm < 4 || warps_per_sm > 64 || warps_per_sm % 4 != 0)
        return set_error(SAQ_ERR_INVALID, "warps_per_sm must be 4, 8, ..., 64");
    if (bits < 1 || bits > 8) return set_error(SAQ_ERR_INVALID, "bits outside 1..8");
    return step_ceiling(warps_per_sm, bits, lane_steps_per_s);
}

saq_status saq_estimate_staged(const saq_model *m, const uint8_t *codes_dev,
                               const float *factors_dev, int64_t n, const float *Q_dev, int64_t nq,
                               float m_conf, float *bounds_dev, void *stream) {
    clear_error();
    if (!m) return set_error(SAQ_ERR_INVALID, "model is NULL");
    if (n < 0 || nq < 0) return set_error(SAQ_ERR_INVALID, "negative size");
    if (!(m_conf >= 0.f) || !std::isfinite(m_conf))
        return set_error(SAQ_ERR_INVALID, "m must be finite and >= 0");
    if (m->Vt.empty() || !m->d_B)
        return set_error(SAQ_ERR_UNSUPPORTED,
                         "the model carries no PCA basis (saq_fit sets it; see saq_model_set_basis)");
    if (n == 0 || nq == 0) return SAQ_OK;
    if (n * nq > ((int64_t)1 << 33)) return set_error(SAQ_ERR_UNSUPPORTED, "n * nq too large");
    if (!factors_dev || !Q_dev || !bounds_dev || (m->code_bytes > 0 && !codes_dev))
        return set_error(SAQ_ERR_INVALID, "NULL buffer");
    if (!aligned16(codes_dev) || !aligned16(factors_dev) || !aligned16(Q_dev))
        return set_error(SAQ_ERR_INVALID, "device buffers must be 16-byte aligned");
    saq_status st = check_device(m);
    if (st != SAQ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nk = std::max<size_t>(1, m->kept.size());
    float *qrot = nullptr, *qn2 = nullptr, *vs = nullptr, *qsig = nullptr;
    const size_t bq = sizeof(float) * (size_t)nq * std::max(1, m->dk);
    if (scratch_alloc((void **)&qrot, bq, s) != cudaSuccess ||
        scratch_alloc((void **)&qn2, sizeof(float) * (size_t)nq, s) != cudaSuccess ||
        scratch_alloc((void **)&vs, sizeof(float) * (size_t)n * nk, s) != cudaSuccess ||
        scratch_alloc((void **)&qsig, sizeof(float) * (size_t)nq * nk, s) != cudaSuccess) {
        if (qrot) cudaFreeAsync(qrot, s);
        if (qn2) cudaFreeAsync(qn2, s);
        if (vs) cudaFreeAsync(vs, s);
        return set_error(SAQ_ERR_OOM, "scratch allocation failed");
    }
    st = launch_project_simt(m, Q_dev, nq, qrot, m->dk, kRowMajor, s);
    if (st == SAQ_OK) st = launch_rownorm2(m, Q_dev, nq, qn2, 1, s);
    if (st == SAQ_OK)
        st = launch_estimate_staged(m, codes_dev, factors_dev, n, Q_dev, qrot, qn2, nq, m_conf, vs,
                                    qsig, bounds_dev, s);
    cudaFreeAsync(qrot, s);
    cudaFreeAsync(qn2, s);
    cudaFreeAsync(vs, s);
    cudaFreeAsync(qsig, s);
    return st;
}

}  // extern "C"
