// saq_ingest.cu -- serving runtime: continuous batching of insert requests
// over several resident collections (see include/saq.h).
//
// Host side only; the device work of a batch is the encode of saq_encode
// (projection + quantize/adjust/pack kernels) on the batch's slot stream,
// between an H2D copy per request piece and a D2H copy per piece.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "saq_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int coll = 0;
    const float *X = nullptr;
    int64_t n = 0;
    uint8_t *codes = nullptr;
    float *factors = nullptr;
    int64_t next_row = 0;   // rows handed to batches
    int64_t rows_done = 0;  // rows whose outputs are in host memory
    bool done = false;
    saq_status status = SAQ_OK;
    Clock::time_point t_submit, t_done;
};

struct Piece {
    Request *req;
    int64_t r0, nr, off;  // rows [r0, r0 + nr) of req at batch row `off`
};

struct Slot {
    cudaStream_t stream = nullptr;
    float *X = nullptr, *factors = nullptr;
    void *O = nullptr;
    uint8_t *codes = nullptr;
    int *err_dev = nullptr;   // the batch's device error word (bounded waits, input range)
    int *err_host = nullptr;  // its copy, written on the slot stream before the callback
    bool busy = false;
    bool finished = false;  // set by the stream callback
    std::vector<Piece> pieces;
};

}  // namespace

struct saq_ingest {
    std::vector<saq_model *> models;
    saq_ingest_params p{};
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::vector<std::deque<Request *>> queues;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread th;
    // statistics
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, rows_completed = 0, batches = 0;
    double max_lat = 0;
    bool any_submit = false;
    Clock::time_point t_first, t_last;
};

namespace {

using saq::set_error;

void CUDART_CB on_batch_done(void *arg) {
    // runs on a CUDA callback thread: no CUDA calls here
    auto *pr = static_cast<std::pair<saq_ingest *, Slot *> *>(arg);
    saq_ingest *s = pr->first;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        pr->second->finished = true;
    }
    s->cv_sched.notify_one();
    delete pr;
}

// Complete the batches whose stream callback fired.  Caller holds mu.
void reap(saq_ingest *s) {
    for (Slot &sl : s->slots) {
        if (!sl.busy || !sl.finished) continue;
        // the callback fired, so the batch's copies and kernels are done; the
        // callback itself may still be returning (not-ready is no error)
        const cudaError_t e = cudaStreamQuery(sl.stream);
        const bool failed = e != cudaSuccess && e != cudaErrorNotReady;
        // a wait of the batch's projection that gave up, or an input row out
        // of range, fails every request with rows in the batch
        const saq_status dev_st = *sl.err_host ? saq::tc_error_status(*sl.err_host) : SAQ_OK;
        *sl.err_host = 0;
        const Clock::time_point now = Clock::now();
        for (const Piece &pc : sl.pieces) {
            Request *r = pc.req;
            if (failed) r->status = SAQ_ERR_CUDA;
            else if (dev_st != SAQ_OK && r->status == SAQ_OK) r->status = dev_st;
            r->rows_done += pc.nr;
            if (r->rows_done == r->n && !r->done) {
                r->done = true;
                r->t_done = now;
                const double l = std::chrono::duration<double>(now - r->t_submit).count();
                s->lat.push_back(l);
                s->max_lat = std::max(s->max_lat, l);
                s->completed += 1;
                s->rows_completed += (uint64_t)r->n;
                s->t_last = now;
            }
        }
        sl.pieces.clear();
        sl.busy = false;
        sl.finished = false;
    }
    s->cv_done.notify_all();
}

// Pick the collection whose oldest queued request is the oldest overall.
int pick_collection(saq_ingest *s) {
    int best = -1;
    Clock::time_point t{};
    for (size_t c = 0; c < s->queues.size(); ++c) {
        if (s->queues[c].empty()) continue;
        const Clock::time_point tc = s->queues[c].front()->t_submit;
        if (best < 0 || tc < t) { best = (int)c; t = tc; }
    }
    return best;
}

// Form a batch for a free slot and enqueue its work.  Caller holds mu.
void dispatch(saq_ingest *s, Slot &sl, int coll) {
    saq_model *m = s->models[(size_t)coll];
    std::deque<Request *> &q = s->queues[(size_t)coll];
    int64_t rows = 0;
    const int64_t cap = s->p.max_batch_rows;
    while (!q.empty() && rows < cap) {
        Request *r = q.front();
        const int64_t k = std::min(r->n - r->next_row, cap - rows);
        sl.pieces.push_back(Piece{r, r->next_row, k, rows});
        r->next_row += k;
        rows += k;
        if (r->next_row == r->n) q.pop_front();
    }
    sl.busy = true;
    sl.finished = false;
    s->batches += 1;
    const int d = m->d;
    const size_t cb = m->code_bytes;
    const int nf = m->nf;
    saq_status st = SAQ_OK;
    for (const Piece &pc : sl.pieces)
        if (cudaMemcpyAsync(sl.X + pc.off * d, pc.req->X + pc.r0 * d, sizeof(float) * (size_t)pc.nr * d,
                            cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            st = SAQ_ERR_CUDA;
    if (st == SAQ_OK) {
        if (m->dk == 0) st = saq::launch_rownorm2(m, sl.X, rows, sl.factors, nf, sl.stream);
        else st = saq::encode_rows(m, sl.X, rows, sl.codes, sl.factors, sl.O, cap, sl.stream,
                                   sl.err_dev);
    }
    if (st == SAQ_OK && (cudaMemcpyAsync(sl.err_host, sl.err_dev, sizeof(int),
                                         cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                         cudaMemsetAsync(sl.err_dev, 0, sizeof(int), sl.stream) != cudaSuccess))
        st = SAQ_ERR_CUDA;
    for (const Piece &pc : sl.pieces) {
        if (cb)
            cudaMemcpyAsync(pc.req->codes + pc.r0 * (int64_t)cb, sl.codes + pc.off * (int64_t)cb,
                            cb * (size_t)pc.nr, cudaMemcpyDeviceToHost, sl.stream);
        cudaMemcpyAsync(pc.req->factors + pc.r0 * nf, sl.factors + pc.off * nf,
                        sizeof(float) * (size_t)pc.nr * nf, cudaMemcpyDeviceToHost, sl.stream);
        if (st != SAQ_OK) pc.req->status = st;
    }
    auto *arg = new std::pair<saq_ingest *, Slot *>(s, &sl);
    if (cudaLaunchHostFunc(sl.stream, on_batch_done, arg) != cudaSuccess) {
        delete arg;
        for (const Piece &pc : sl.pieces) pc.req->status = SAQ_ERR_CUDA;
        cudaStreamSynchronize(sl.stream);
        sl.finished = true;
    }
}

void scheduler(saq_ingest *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap(s);
        for (Slot &sl : s->slots) {
            if (sl.busy) continue;
            const int c = pick_collection(s);
            if (c < 0) break;
            dispatch(s, sl, c);
        }
        bool busy = false, queued = false;
        for (Slot &sl : s->slots) busy |= sl.busy;
        for (auto &q : s->queues) queued |= !q.empty();
        if (s->stopping && !busy && !queued) break;
        bool ready = false;
        for (Slot &sl : s->slots) ready |= (sl.busy && sl.finished);
        if (ready) continue;
        bool free_slot = false;
        for (Slot &sl : s->slots) free_slot |= !sl.busy;
        if (queued && free_slot) continue;
        s->cv_sched.wait(lk);
    }
}

void free_slots(saq_ingest *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        cudaFree(sl.X);
        cudaFree(sl.codes);
        cudaFree(sl.factors);
        cudaFree(sl.O);
        cudaFree(sl.err_dev);
        if (sl.err_host) cudaFreeHost(sl.err_host);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

saq_status saq_ingest_open(saq_model *const *models, int32_t n_models,
                           const saq_ingest_params *p, saq_ingest **out) {
    saq::clear_error();
    if (!out) return set_error(SAQ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!models || n_models < 1 || !p) return set_error(SAQ_ERR_INVALID, "no collections");
    if (p->max_batch_rows < 1 || p->slots < 1 || p->slots > 64)
        return set_error(SAQ_ERR_INVALID, "max_batch_rows >= 1 and 1 <= slots <= 64 required");
    int dev = 0;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    int dmax = 0, dkmax = 0, nfmax = 0;
    size_t cbmax = 0, scrmax = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        if (!models[i]) return set_error(SAQ_ERR_INVALID, "collection %d is NULL", i);
        if (models[i]->device != dev)
            return set_error(SAQ_ERR_INVALID, "collection %d lives on another device", i);
        dmax = std::max(dmax, models[i]->d);
        dkmax = std::max(dkmax, models[i]->dk);
        nfmax = std::max(nfmax, models[i]->nf);
        cbmax = std::max(cbmax, models[i]->code_bytes);
        scrmax = std::max(scrmax, saq::encode_scratch_bytes(models[i], p->max_batch_rows));
    }
    const size_t rows = (size_t)p->max_batch_rows;
    const size_t per_slot = rows * (sizeof(float) * ((size_t)dmax + nfmax) + cbmax) + scrmax +
                            4 * 256;
    if (per_slot * (size_t)p->slots > p->hbm_budget_bytes)
        return set_error(SAQ_ERR_OOM,
                         "%d slots of %zu bytes exceed the HBM budget of %zu bytes", p->slots,
                         per_slot, p->hbm_budget_bytes);
    saq_ingest *s = new (std::nothrow) saq_ingest();
    if (!s) return set_error(SAQ_ERR_OOM, "host allocation failed");
    s->models.assign(models, models + n_models);
    s->p = *p;
    s->device = dev;
    s->queues.resize((size_t)n_models);
    s->slots.resize((size_t)p->slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&sl.X, sizeof(float) * rows * dmax) != cudaSuccess ||
            cudaMalloc(&sl.codes, std::max<size_t>(16, cbmax * rows)) != cudaSuccess ||
            cudaMalloc(&sl.factors, sizeof(float) * rows * nfmax) != cudaSuccess ||
            cudaMalloc(&sl.O, scrmax) != cudaSuccess ||
            cudaMalloc(&sl.err_dev, sizeof(int)) != cudaSuccess ||
            cudaMemset(sl.err_dev, 0, sizeof(int)) != cudaSuccess ||
            cudaHostAlloc(&sl.err_host, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            free_slots(s);
            delete s;
            return set_error(SAQ_ERR_OOM, "slot allocation failed");
        }
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return SAQ_OK;
}

saq_status saq_ingest_submit(saq_ingest *s, int32_t collection, const float *X_host, int64_t n,
                             uint8_t *codes_host, float *factors_host, uint64_t *ticket) {
    saq::clear_error();
    if (!s || !ticket) return set_error(SAQ_ERR_INVALID, "NULL argument");
    if (collection < 0 || collection >= (int32_t)s->models.size())
        return set_error(SAQ_ERR_INVALID, "no collection %d", collection);
    if (n < 1 || !X_host || !factors_host ||
        (s->models[(size_t)collection]->code_bytes > 0 && !codes_host))
        return set_error(SAQ_ERR_INVALID, "empty request or NULL buffer");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(SAQ_ERR_OOM, "host allocation failed");
    r->coll = collection;
    r->X = X_host;
    r->n = n;
    r->codes = codes_host;
    r->factors = factors_host;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete r;
            return set_error(SAQ_ERR_INVALID, "service is closing");
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queues[(size_t)collection].push_back(r);
        s->submitted += 1;
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first = r->t_submit;
        }
        *ticket = r->ticket;
    }
    s->cv_sched.notify_one();
    return SAQ_OK;
}

saq_status saq_ingest_poll(saq_ingest *s, uint64_t ticket, int32_t *done) {
    if (!s || !done) return set_error(SAQ_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAQ_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->done ? 1 : 0;
    return it->second->done ? it->second->status : SAQ_OK;
}

saq_status saq_ingest_wait(saq_ingest *s, uint64_t ticket, int32_t timeout_ms, double *latency_s) {
    if (!s) return set_error(SAQ_ERR_INVALID, "NULL service");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAQ_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto pred = [r]() { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return set_error(SAQ_ERR_TIMEOUT, "request %llu still in flight", (unsigned long long)ticket);
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    const saq_status st = r->status;
    s->reqs.erase(it);
    delete r;
    if (st != SAQ_OK)
        return set_error(st, "request failed on the device: %s", saq_status_string(st));
    return SAQ_OK;
}

saq_status saq_ingest_get_stats(saq_ingest *s, saq_ingest_stats *out) {
    if (!s || !out) return set_error(SAQ_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rows_completed = s->rows_completed;
    out->batches = s->batches;
    out->max_latency_s = s->max_lat;
    std::vector<double> v = s->lat;
    auto q = [&v](double f) {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + (long)k, v.end());
        return v[k];
    };
    out->p50_latency_s = q(0.50);
    out->p99_latency_s = q(0.99);
    out->busy_s = s->completed ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    return SAQ_OK;
}

saq_status saq_ingest_close(saq_ingest *s) {
    if (!s) return SAQ_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_sched.notify_one();
    if (s->th.joinable()) s->th.join();
    free_slots(s);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return SAQ_OK;
}

}  // extern "C"
