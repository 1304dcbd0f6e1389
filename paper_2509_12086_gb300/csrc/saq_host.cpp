// saq_host.cpp -- host side of the library: error state, parameters, the
// plan search (Algorithm 2), the rotation RNG, and model construction,
// queries and serialisation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>
#include <mutex>
#include <vector>

#include "saq_internal.h"

namespace saq {

static thread_local std::string g_last_error;

saq_status set_error(saq_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

void clear_error() { g_last_error.clear(); }

static std::atomic<uint64_t> g_launches{0};
void note_launches(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pool[dev], &props);
            if (e != cudaSuccess) {
                g_pool[dev] = nullptr;
                return e;
            }
            // without a threshold the pool unmaps its memory at every
            // synchronisation, and the next call maps it again
            uint64_t keep = kPoolKeepBytes;
            cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

namespace {
struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};
std::atomic<int> g_timing{0};
std::mutex g_timing_mu;
std::vector<TimedLaunch> g_timed;
}  // namespace

LaunchTimer::LaunchTimer(int k, cudaStream_t st) : kind(k), s(st) {
    if (!g_timing.load(std::memory_order_relaxed)) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        a = nullptr;
    }
}
LaunchTimer::~LaunchTimer() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, s) != cudaSuccess) {
        if (b) cudaEventDestroy(b);
        cudaEventDestroy(a);
        return;
    }
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timed.push_back(TimedLaunch{kind, a, b});
}

// ------------------------------------------------------------------------
// Quantization plan search, Sec. 4.2 Algorithm 2.
//
// Modelled error of a segment: sum of sigma_i^2 over the segment times 2^-B
// (Eq. seg-err, empirical-variance form without pi; B = 0 drops the segment
// at its full variance).  Segment boundaries lie on multiples of g (plus D),
// bits range over 0..max_bits, and the plan's cost B*|Seg| summed must stay
// within the quota.  best[pos][q][k] holds the least error of plans that
// cover the first grid positions `pos` with exactly q cost units and k
// segments; states are visited in the order pos, q, k, next boundary, bits,
// and replaced only on a strictly smaller error.  The returned plan has the
// fewest segments among plans within (1 + tie_frac) of the least error, then
// the least error, then the least cost.
// ------------------------------------------------------------------------
int plan_search(const double *sig2, int D, int g, int64_t quota_bits,
                int max_bits, double tie_frac, std::vector<saq_segment> &out,
                double *err, double *min_err) {
    if (D < 1 || g < 1 || max_bits < 0 || max_bits > 8 || quota_bits < 0)
        return -1;
    std::vector<int> grid;
    for (int x = 0; x < D; x += g) grid.push_back(x);
    grid.push_back(D);
    const int P = (int)grid.size();
    int64_t unit = g;
    if (D % g) {
        int64_t a = g, b = D % g;
        while (b) { int64_t t = a % b; a = b; b = t; }
        unit = a;
    }
    const int64_t Qn = quota_bits / unit + 1;
    std::vector<double> cum(D + 1, 0.0);
    for (int i = 0; i < D; ++i) cum[i + 1] = cum[i] + sig2[i];

    struct Cell { double e; int from; int64_t fq; int b; };
    const double INF = std::numeric_limits<double>::infinity();
    const size_t cells = (size_t)P * (size_t)Qn * (size_t)P;
    std::vector<Cell> best;
    try {
        best.assign(cells, Cell{INF, -1, -1, -1});
    } catch (...) {
        return -1;
    }
    auto at = [&](int pos, int64_t q, int k) -> Cell & {
        return best[((size_t)pos * (size_t)Qn + (size_t)q) * (size_t)P + (size_t)k];
    };
    at(0, 0, 0).e = 0.0;
    for (int pos = 0; pos + 1 < P; ++pos)
        for (int64_t q = 0; q < Qn; ++q)
            for (int k = 0; k <= pos; ++k) {
                const double base = at(pos, q, k).e;
                if (base == INF) continue;
                for (int nxt = pos + 1; nxt < P; ++nxt) {
                    const int len = grid[nxt] - grid[pos];
                    const double var = cum[grid[nxt]] - cum[grid[pos]];
                    for (int b = 0; b <= max_bits; ++b) {
                        const int64_t q2 = q + (int64_t)b * len / unit;
                        if (q2 >= Qn) break;
                        const double e = base + ldexp(var, -b);
                        Cell &c = at(nxt, q2, k + 1);
                        if (e < c.e) c = Cell{e, pos, q, b};
                    }
                }
            }
    const int last = P - 1;
    double emin = INF;
    for (int64_t q = 0; q < Qn; ++q)
        for (int k = 1; k < P; ++k) emin = std::min(emin, at(last, q, k).e);
    if (emin == INF) return -1;
    const double limit = emin * (1.0 + tie_frac);
    int kb = -1;
    int64_t qb = -1;
    double eb = INF;
    for (int k = 1; k < P && kb < 0; ++k) {
        for (int64_t q = 0; q < Qn; ++q) {
            const double e = at(last, q, k).e;
            if (e <= limit && e < eb) { eb = e; qb = q; }
        }
        if (qb >= 0) kb = k;
    }
    out.assign((size_t)kb, saq_segment{0, 0, 0});
    int pos = last;
    int64_t q = qb;
    for (int k = kb; k > 0; --k) {
        const Cell &c = at(pos, q, k);
        out[(size_t)k - 1] = saq_segment{grid[c.from], grid[pos] - grid[c.from], c.b};
        pos = c.from;
        q = c.fq;
    }
    *err = eb;
    *min_err = emin;
    return 0;
}

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.
// Draw i uses counter (i/2, stream_lo, stream_hi, 0) and key (seed_lo,
// seed_hi); two 53-bit uniforms in (0, 1) give a Gaussian pair.
// ------------------------------------------------------------------------
static inline void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * c[0];
        const uint64_t p1 = (uint64_t)M1 * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

void philox_gaussian(uint64_t seed, uint64_t stream_id, double *out, size_t n) {
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0;
    for (size_t i = 0; i < n; i += 2) {
        uint32_t c[4] = {(uint32_t)(i / 2), (uint32_t)((i / 2) >> 32) ^ (uint32_t)stream_id,
                         (uint32_t)(stream_id >> 32), 0x5A51u};
        philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u1 = ((double)((uint64_t)(c[0] >> 5) * 67108864ull + (c[1] >> 6)) + 0.5) * inv53;
        const double u2 = ((double)((uint64_t)(c[2] >> 5) * 67108864ull + (c[3] >> 6)) + 0.5) * inv53;
        const double r = sqrt(-2.0 * log(u1));
        out[i] = r * cos(two_pi * u2);
        if (i + 1 < n) out[i + 1] = r * sin(two_pi * u2);
    }
}

// ------------------------------------------------------------------------
// Model construction
// ------------------------------------------------------------------------
void model_release_device(saq_model *m) {
    if (!m) return;
    cudaFree(m->d_mean);
    cudaFree(m->d_W);
    cudaFree(m->d_B);
    m->d_B = nullptr;
    tc_release(m);
    m->d_mean = nullptr;
    m->d_W = nullptr;
}

saq_status model_finalize(saq_model *m) {
    m->kept.clear();
    int off = 0, fidx = 1;
    int64_t cb = 0;
    for (const saq_segment &s : m->plan) {
        if (s.bits == 0) continue;
        KeptSeg k;
        k.start = s.start;
        k.off = off;
        k.len = s.len;
        k.bits = s.bits;
        k.words = (s.len + 63) / 64;
        k.code_off = cb;
        k.fidx = fidx;
        m->kept.push_back(k);
        off += s.len;
        cb += (int64_t)s.bits * k.words * 8;
        fidx += 2;
    }
    m->dk = off;
    m->code_bytes = (size_t)cb;
    m->nf = fidx;
    SAQ_CUDA_CHECK(cudaGetDevice(&m->device));
    std::vector<float> f(m->mean.begin(), m->mean.end());
    SAQ_CUDA_CHECK(cudaMalloc(&m->d_mean, sizeof(float) * (size_t)std::max(1, m->d)));
    SAQ_CUDA_CHECK(cudaMemcpy(m->d_mean, f.data(), sizeof(float) * (size_t)m->d,
                              cudaMemcpyHostToDevice));
    if (m->dk > 0) {
        std::vector<float> w(m->W.begin(), m->W.end());
        SAQ_CUDA_CHECK(cudaMalloc(&m->d_W, sizeof(float) * w.size()));
        SAQ_CUDA_CHECK(cudaMemcpy(m->d_W, w.data(), sizeof(float) * w.size(),
                                  cudaMemcpyHostToDevice));
    }
    // the tensor-core forms take d % 4 == 0 and d <= 6144; another d needs
    // the CUDA-core projection, chosen explicitly (no silent switch)
    if (m->precision != SAQ_PREC_FP32_SIMT && m->dk > 0 && !tc_supported(m))
        return set_error(SAQ_ERR_UNSUPPORTED,
                         "the tensor-core projection needs d %% 4 == 0 and d <= 6144 (d = %d); "
                         "use SAQ_PREC_FP32_SIMT for this model", m->d);
    if (m->precision != SAQ_PREC_FP32_SIMT && tc_supported(m)) {
        saq_status st = model_build_tc(m, m->precision, 0);
        if (st != SAQ_OK) return st;
        SAQ_CUDA_CHECK(cudaDeviceSynchronize());
    }
    return SAQ_OK;
}

saq_status model_upload_basis(saq_model *m) {
    cudaFree(m->d_B);
    m->d_B = nullptr;
    if (m->Vt.empty() || m->dk == 0) return SAQ_OK;
    // row i of the kept dimensions: sigma_i v_i^T, sigma_i of its PCA dimension
    std::vector<float> b(m->Vt.size());
    int row = 0;
    for (const saq::KeptSeg &k : m->kept)
        for (int r = 0; r < k.len; ++r, ++row) {
            const double sg = sqrt(std::max(0.0, m->sig2[(size_t)(k.start + r)]));
            for (int j = 0; j < m->d; ++j)
                b[(size_t)row * m->d + j] = (float)(sg * m->Vt[(size_t)row * m->d + j]);
        }
    SAQ_CUDA_CHECK(cudaMalloc(&m->d_B, sizeof(float) * b.size()));
    SAQ_CUDA_CHECK(cudaMemcpy(m->d_B, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice));
    return SAQ_OK;
}

static saq_status check_plan(int32_t d, const saq_segment *plan, int32_t nseg) {
    if (!plan || nseg < 1) return set_error(SAQ_ERR_INVALID, "empty plan");
    int32_t at = 0;
    for (int32_t i = 0; i < nseg; ++i) {
        if (plan[i].start != at || plan[i].len < 1)
            return set_error(SAQ_ERR_INVALID, "plan segment %d does not continue at %d", i, at);
        if (plan[i].bits < 0 || plan[i].bits > 8)
            return set_error(SAQ_ERR_INVALID, "plan segment %d: bits %d outside 0..8", i,
                             plan[i].bits);
        at += plan[i].len;
    }
    if (at != d) return set_error(SAQ_ERR_INVALID, "plan covers %d of %d dimensions", at, d);
    return SAQ_OK;
}

}  // namespace saq

using namespace saq;

extern "C" {

void saq_params_init(saq_params *p) {
    if (!p) return;
    p->avg_bits = 4.0;
    p->max_bits = 8;
    p->rounds = 6;
    p->seg_granularity = 64;
    p->precision = SAQ_PREC_FP32;
    p->tie_frac = 1e-3;
    p->seed = 4;
}

const char *saq_last_error(void) { return g_last_error.c_str(); }

uint64_t saq_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

saq_status saq_kernel_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!enable) {  // stop; the record stays readable
        g_timing.store(0);
        return SAQ_OK;
    }
    for (const TimedLaunch &t : g_timed) {
        cudaEventSynchronize(t.b);
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_timed.clear();
    g_timing.store(1);
    return SAQ_OK;
}

saq_status saq_kernel_times(double *ms, int64_t *launches, int kinds) {
    if (!ms || !launches || kinds < 1 || kinds > kKindCount)
        return set_error(SAQ_ERR_INVALID, "saq_kernel_times: need host arrays of 1..%d kinds", kKindCount);
    for (int k = 0; k < kinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (const TimedLaunch &t : g_timed) {
        float e = 0.f;
        SAQ_CUDA_CHECK(cudaEventSynchronize(t.b));
        SAQ_CUDA_CHECK(cudaEventElapsedTime(&e, t.a, t.b));
        if (t.kind < kinds) {
            ms[t.kind] += e;
            launches[t.kind] += 1;
        }
    }
    return SAQ_OK;
}

saq_status saq_plan_search(const double *sig2, int32_t d, int32_t g, int64_t quota_bits,
                           int32_t max_bits, double tie_frac, saq_segment *out, int32_t cap,
                           int32_t *nseg, double *err) {
    clear_error();
    if (!sig2 || !out || !nseg || d < 1 || g < 1 || quota_bits < 0 || max_bits < 0 ||
        max_bits > 8 || !(tie_frac >= 0.0))
        return set_error(SAQ_ERR_INVALID, "bad plan-search arguments");
    std::vector<saq_segment> plan;
    double e = 0, emin = 0;
    if (plan_search(sig2, d, g, quota_bits, max_bits, tie_frac, plan, &e, &emin) != 0)
        return set_error(SAQ_ERR_OOM, "plan search failed");
    if ((int32_t)plan.size() > cap) return set_error(SAQ_ERR_INVALID, "cap too small");
    std::copy(plan.begin(), plan.end(), out);
    *nseg = (int32_t)plan.size();
    if (err) *err = e;
    return SAQ_OK;
}

const char *saq_status_string(saq_status s) {
    switch (s) {
        case SAQ_OK: return "ok";
        case SAQ_ERR_INVALID: return "invalid argument";
        case SAQ_ERR_CUDA: return "CUDA error";
        case SAQ_ERR_OOM: return "out of memory";
        case SAQ_ERR_TIMEOUT: return "device wait timed out";
        case SAQ_ERR_UNSUPPORTED: return "unsupported";
        case SAQ_ERR_RANGE: return "input out of range";
    }
    return "unknown status";
}

saq_status saq_model_create(int32_t d, const double *mean, const double *W,
                            const saq_segment *plan, int32_t nseg,
                            const double *sig2, const saq_params *p,
                            saq_model **out) {
    clear_error();
    if (!out) return set_error(SAQ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (d < 1 || !mean || !p) return set_error(SAQ_ERR_INVALID, "d < 1 or NULL mean/params");
    saq_status st = check_plan(d, plan, nseg);
    if (st != SAQ_OK) return st;
    if (p->rounds < 0 || p->rounds > 1000)
        return set_error(SAQ_ERR_INVALID, "rounds %d outside 0..1000", p->rounds);
    if (p->precision < 0 || p->precision > 3)
        return set_error(SAQ_ERR_INVALID, "unknown precision %d", p->precision);
    int64_t dk = 0;
    for (int32_t i = 0; i < nseg; ++i)
        if (plan[i].bits > 0) dk += plan[i].len;
    if (dk > 0 && !W) return set_error(SAQ_ERR_INVALID, "W is NULL");
    saq_model *m = new (std::nothrow) saq_model();
    if (!m) return set_error(SAQ_ERR_OOM, "host allocation failed");
    m->d = d;
    m->rounds = p->rounds;
    m->precision = p->precision;
    m->plan.assign(plan, plan + nseg);
    m->mean.assign(mean, mean + d);
    if (dk > 0) m->W.assign(W, W + dk * (int64_t)d);
    if (sig2) m->sig2.assign(sig2, sig2 + d);
    else m->sig2.assign((size_t)d, 0.0);
    st = model_finalize(m);
    if (st != SAQ_OK) {
        model_release_device(m);
        delete m;
        return st;
    }
    *out = m;
    return SAQ_OK;
}

void saq_model_free(saq_model *m) {
    if (!m) return;
    model_release_device(m);
    delete m;
}

size_t saq_code_bytes(const saq_model *m) { return m ? m->code_bytes : 0; }
int32_t saq_factor_count(const saq_model *m) { return m ? m->nf : 0; }
int32_t saq_model_dim(const saq_model *m) { return m ? m->d : 0; }
int32_t saq_model_kept_dim(const saq_model *m) { return m ? m->dk : 0; }
int32_t saq_model_num_segments(const saq_model *m) { return m ? (int32_t)m->plan.size() : 0; }

saq_status saq_model_get_plan(const saq_model *m, saq_segment *out, int32_t cap) {
    if (!m || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    if (cap < (int32_t)m->plan.size()) return set_error(SAQ_ERR_INVALID, "cap too small");
    std::copy(m->plan.begin(), m->plan.end(), out);
    return SAQ_OK;
}

saq_status saq_model_get_mean(const saq_model *m, double *out) {
    if (!m || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    std::copy(m->mean.begin(), m->mean.end(), out);
    return SAQ_OK;
}

saq_status saq_model_get_matrix(const saq_model *m, double *out) {
    if (!m || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    std::copy(m->W.begin(), m->W.end(), out);
    return SAQ_OK;
}

saq_status saq_model_get_variances(const saq_model *m, double *out) {
    if (!m || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    std::copy(m->sig2.begin(), m->sig2.end(), out);
    return SAQ_OK;
}

saq_status saq_model_set_basis(saq_model *m, const double *Vt) {
    clear_error();
    if (!m || !Vt) return set_error(SAQ_ERR_INVALID, "NULL argument");
    for (int64_t i = 0; i < (int64_t)m->dk * m->d; ++i)
        if (!std::isfinite(Vt[i])) return set_error(SAQ_ERR_INVALID, "basis has a non-finite entry");
    m->Vt.assign(Vt, Vt + (int64_t)m->dk * m->d);
    return model_upload_basis(m);
}

int32_t saq_model_has_basis(const saq_model *m) { return m && !m->Vt.empty() ? 1 : 0; }

saq_status saq_model_set_rounds(saq_model *m, int32_t rounds) {
    if (!m || rounds < 0 || rounds > 1000)
        return set_error(SAQ_ERR_INVALID, "bad model or rounds");
    m->rounds = rounds;
    return SAQ_OK;
}

saq_status saq_model_set_precision(saq_model *m, int32_t precision) {
    clear_error();
    if (!m || precision < 0 || precision > 3)
        return set_error(SAQ_ERR_INVALID, "bad model or precision");
    // checked before anything changes: a refused precision leaves the model as it was
    if (precision != SAQ_PREC_FP32_SIMT && m->dk > 0 && !tc_supported(m))
        return set_error(SAQ_ERR_UNSUPPORTED,
                         "the tensor-core projection needs d %% 4 == 0 and d <= 6144 (d = %d); "
                         "use SAQ_PREC_FP32_SIMT for this model", m->d);
    m->precision = precision;
    if (precision == SAQ_PREC_FP32_SIMT || m->dk == 0) return SAQ_OK;
    saq_status st = model_build_tc(m, precision, 0);
    if (st != SAQ_OK) return st;
    SAQ_CUDA_CHECK(cudaDeviceSynchronize());
    return SAQ_OK;
}

// Blob: "SAQM" u32 version, i32 d, i32 nseg, i32 rounds, i32 precision,
// nseg x (i32 start, i32 len, i32 bits), d x f64 mean, d x f64 sig2,
// dk x d x f64 W; version 2 adds i32 has_basis and, if set, dk x d x f64 Vt.
// Little-endian (host order on every supported host).  Import reads 1 and 2.
static const uint32_t kVersion = 2;

saq_status saq_model_export(const saq_model *m, void *buf, size_t *len) {
    if (!m || !len) return set_error(SAQ_ERR_INVALID, "NULL argument");
    const size_t need = 4 + 4 + 4 * 4 + m->plan.size() * 12 + (size_t)m->d * 16 +
                        m->W.size() * 8 + 4 + m->Vt.size() * 8;
    if (!buf) { *len = need; return SAQ_OK; }
    if (*len < need) return set_error(SAQ_ERR_INVALID, "buffer too small (%zu < %zu)", *len, need);
    uint8_t *p = (uint8_t *)buf;
    auto put = [&](const void *src, size_t n) { memcpy(p, src, n); p += n; };
    put("SAQM", 4);
    put(&kVersion, 4);
    int32_t hdr[4] = {m->d, (int32_t)m->plan.size(), m->rounds, m->precision};
    put(hdr, sizeof(hdr));
    for (const saq_segment &s : m->plan) {
        int32_t v[3] = {s.start, s.len, s.bits};
        put(v, 12);
    }
    put(m->mean.data(), (size_t)m->d * 8);
    put(m->sig2.data(), (size_t)m->d * 8);
    put(m->W.data(), m->W.size() * 8);
    const int32_t hb = m->Vt.empty() ? 0 : 1;
    put(&hb, 4);
    if (hb) put(m->Vt.data(), m->Vt.size() * 8);
    *len = need;
    return SAQ_OK;
}

saq_status saq_model_import(const void *buf, size_t len, saq_model **out) {
    clear_error();
    if (!buf || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    const uint8_t *p = (const uint8_t *)buf;
    if (len < 24 || memcmp(p, "SAQM", 4) != 0)
        return set_error(SAQ_ERR_INVALID, "not a model blob");
    uint32_t ver;
    memcpy(&ver, p + 4, 4);
    if (ver != 1 && ver != 2) return set_error(SAQ_ERR_INVALID, "blob version %u unsupported", ver);
    int32_t hdr[4];
    memcpy(hdr, p + 8, 16);
    const int32_t d = hdr[0], nseg = hdr[1];
    if (d < 1 || nseg < 1 || nseg > d) return set_error(SAQ_ERR_INVALID, "corrupt header");
    size_t at = 24;
    if (len < at + (size_t)nseg * 12) return set_error(SAQ_ERR_INVALID, "truncated blob");
    std::vector<saq_segment> plan((size_t)nseg);
    for (int32_t i = 0; i < nseg; ++i) {
        int32_t v[3];
        memcpy(v, p + at, 12);
        at += 12;
        plan[(size_t)i] = saq_segment{v[0], v[1], v[2]};
    }
    saq_status st = check_plan(d, plan.data(), nseg);
    if (st != SAQ_OK) return st;
    int64_t dk = 0;
    for (auto &s : plan) if (s.bits > 0) dk += s.len;
    const size_t need = at + (size_t)d * 16 + (size_t)dk * (size_t)d * 8;
    if (len < need) return set_error(SAQ_ERR_INVALID, "truncated blob (%zu < %zu)", len, need);
    std::vector<double> mean((size_t)d), sig2((size_t)d), W((size_t)(dk * d));
    memcpy(mean.data(), p + at, (size_t)d * 8);
    at += (size_t)d * 8;
    memcpy(sig2.data(), p + at, (size_t)d * 8);
    at += (size_t)d * 8;
    memcpy(W.data(), p + at, W.size() * 8);
    at += W.size() * 8;
    std::vector<double> Vt;
    if (ver >= 2) {
        if (len < at + 4) return set_error(SAQ_ERR_INVALID, "truncated blob");
        int32_t hb = 0;
        memcpy(&hb, p + at, 4);
        at += 4;
        if (hb) {
            if (len < at + W.size() * 8) return set_error(SAQ_ERR_INVALID, "truncated blob (basis)");
            Vt.resize(W.size());
            memcpy(Vt.data(), p + at, Vt.size() * 8);
        }
    }
    saq_params prm;
    saq_params_init(&prm);
    prm.rounds = hdr[2];
    prm.precision = hdr[3];
    st = saq_model_create(d, mean.data(), W.data(), plan.data(), nseg, sig2.data(), &prm, out);
    if (st == SAQ_OK && !Vt.empty()) {
        st = saq_model_set_basis(*out, Vt.data());
        if (st != SAQ_OK) {
            saq_model_free(*out);
            *out = nullptr;
        }
    }
    return st;
}

}  // extern "C"
