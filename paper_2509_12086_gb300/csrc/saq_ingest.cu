// saq_ingest.cu -- serving runtime: continuous batching of insert requests
// over several resident collections (see include/saq.h).
//
// Host side only.  A batch takes request pieces of up to kMaxGroups
// collections whose models share the tensor-core precision; its device work
// is one H2D copy per piece, ONE projection launch and ONE quantize launch
// over all its collections (encode_grouped), and one D2H copy per piece, on
// the batch's slot stream.  Its device memory (inputs, codes, factors,
// projection scratch) comes from the library's stream-ordered pool when the
// batch is formed and goes back when it completes; a batch is formed only
// if that memory fits in the HBM budget beside the batches in flight.
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
    int group;        // index into the batch's groups
    int64_t r0, nr;   // rows [r0, r0 + nr) of req ...
    int64_t off;      // ... at row `off` of its group
};

// One collection's rows of a batch, and their device regions.
struct Group {
    int coll = 0;
    int64_t rows = 0;
    float *X = nullptr;
    uint8_t *codes = nullptr;
    float *factors = nullptr;
    void *scratch = nullptr;
};

struct Slot {
    cudaStream_t stream = nullptr;
    // the batch's device error word (bounded waits, input range), then the
    // two work counters of its persistent launches
    int *err_dev = nullptr;
    int *err_host = nullptr;  // its copy, written on the slot stream before the callback
    uint8_t *buf = nullptr;   // the batch's device memory (library pool)
    size_t bytes = 0;         // ... as reserved against the budget
    bool busy = false;
    bool finished = false;  // set by the stream callback
    saq_status launch_status = SAQ_OK;  // an enqueue that failed, applied at completion
    std::vector<Piece> pieces;
    std::vector<Group> groups;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes of `rows` rows of model m in a batch.
size_t group_bytes(const saq_model *m, int64_t rows) {
    if (rows <= 0) return 0;
    const size_t r = (size_t)rows;
    return align256(sizeof(float) * r * (size_t)m->d) + align256(m->code_bytes * r) +
           align256(sizeof(float) * r * (size_t)m->nf) +
           (m->dk > 0 ? align256(saq::encode_scratch_bytes(m, rows)) : 0);
}

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
    size_t in_flight = 0;  // device bytes of the batches in flight
    // statistics
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, rows_completed = 0, batches = 0;
    uint64_t mixed = 0, deferred = 0;
    size_t peak = 0;
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
            else if (sl.launch_status != SAQ_OK && r->status == SAQ_OK) r->status = sl.launch_status;
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
        s->in_flight -= sl.bytes;  // the batch's memory went back on its stream
        sl.bytes = 0;
        sl.buf = nullptr;
        sl.pieces.clear();
        sl.groups.clear();
        sl.busy = false;
        sl.finished = false;
        sl.launch_status = SAQ_OK;
    }
    s->cv_done.notify_all();
}

// Whether a model's rows may join a grouped launch: a tensor-core model, or
// one without kept dimensions (only |x - c|^2 is computed for it).  A
// CUDA-core model's batch holds it alone.
bool groupable(const saq_model *m) { return saq::use_tc(m) || m->dk == 0; }

// Form a batch for the free slot `sl` from the queues and reserve its device
// memory against the budget.  Requests are taken in arrival order over all
// collections whose models can share the launch with the oldest request's
// (up to kMaxGroups collections), at most max_batch_rows rows, and only as
// much as the HBM budget leaves beside the batches in flight.  Returns false
// if nothing could be admitted.  Caller holds mu; the slot is marked busy,
// so that its work can be enqueued without the lock (launch_batch).
bool form_batch(saq_ingest *s, Slot &sl) {
    const int nc = (int)s->queues.size();
    // the oldest queued request decides the batch's class
    int c0 = -1;
    for (int c = 0; c < nc; ++c)
        if (!s->queues[(size_t)c].empty() &&
            (c0 < 0 || s->queues[(size_t)c].front()->t_submit <
                           s->queues[(size_t)c0].front()->t_submit))
            c0 = c;
    if (c0 < 0) return false;
    const saq_model *m0 = s->models[(size_t)c0];
    const bool alone = !groupable(m0);  // a CUDA-core model's batch holds it alone
    // the tensor-core precision of the batch, fixed by its first model with
    // kept dimensions (the grouped projection takes one precision)
    int prec = m0->dk > 0 && !alone ? m0->tc.precision : -1;
    const size_t avail = s->p.hbm_budget_bytes > s->in_flight ? s->p.hbm_budget_bytes - s->in_flight : 0;
    const int64_t cap = s->p.max_batch_rows;
    std::vector<int> gidx((size_t)nc, -1);  // collection -> its group in the batch
    int64_t rows = 0;
    size_t bytes = 0;  // of all groups
    while (rows < cap) {
        // the oldest head request among the collections this batch can take
        int c = -1;
        for (int k = 0; k < nc; ++k) {
            if (s->queues[(size_t)k].empty()) continue;
            const saq_model *mk = s->models[(size_t)k];
            if (alone ? k != c0
                      : !groupable(mk) || (mk->dk > 0 && prec >= 0 && mk->tc.precision != prec))
                continue;
            if (gidx[(size_t)k] < 0 && (int)sl.groups.size() == saq::kMaxGroups) continue;
            if (c < 0 || s->queues[(size_t)k].front()->t_submit <
                             s->queues[(size_t)c].front()->t_submit)
                c = k;
        }
        if (c < 0) break;
        saq_model *m = s->models[(size_t)c];
        Request *r = s->queues[(size_t)c].front();
        const int64_t g_rows = gidx[(size_t)c] < 0 ? 0 : sl.groups[(size_t)gidx[(size_t)c]].rows;
        const size_t others = bytes - group_bytes(m, g_rows);
        int64_t k = std::min(r->n - r->next_row, cap - rows);
        // the most rows of this request that fit in the budget
        auto fits = [&](int64_t kk) { return others + group_bytes(m, g_rows + kk) <= avail; };
        bool spent = false;
        if (!fits(k)) {
            int64_t lo = 0, hi = k;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (fits(mid)) lo = mid;
                else hi = mid - 1;
            }
            k = lo;
            spent = true;  // the budget is spent: this is the last piece
        }
        if (k == 0) break;
        if (gidx[(size_t)c] < 0) {
            if (!alone && m->dk > 0) prec = m->tc.precision;
            gidx[(size_t)c] = (int)sl.groups.size();
            Group g;
            g.coll = c;
            sl.groups.push_back(g);
        }
        Group &g = sl.groups[(size_t)gidx[(size_t)c]];
        sl.pieces.push_back(Piece{r, gidx[(size_t)c], r->next_row, k, g.rows});
        r->next_row += k;
        g.rows += k;
        rows += k;
        bytes = others + group_bytes(m, g.rows);
        if (r->next_row == r->n) s->queues[(size_t)c].pop_front();
        if (spent) break;
    }
    if (sl.groups.empty()) {
        s->deferred += 1;
        return false;
    }
    sl.bytes = bytes;
    sl.busy = true;
    sl.finished = false;
    sl.launch_status = SAQ_OK;
    s->in_flight += bytes;
    s->peak = std::max(s->peak, s->in_flight);
    s->batches += 1;
    if (sl.groups.size() > 1) s->mixed += 1;
    return true;
}

// Enqueue a formed batch's work on its slot stream: device memory from the
// pool, one copy-in per piece, the encode of all its collections, the error
// word, one copy-out per piece, the memory back to the pool, and the
// completion callback.  Runs WITHOUT the lock (a copy to or from pageable
// host memory blocks the calling thread until it is done, and submit, wait
// and poll must not wait for that); it touches only the busy slot, the
// immutable parts of the requests and the models.  Returns false if the
// callback could not be enqueued (the stream was synchronised instead).
bool launch_batch(saq_ingest *s, Slot &sl) {
    const size_t bytes = sl.bytes;
    // the batch's device memory, from the pool on the slot stream
    saq_status st = SAQ_OK;
    void *buf = nullptr;
    if (saq::scratch_alloc(&buf, bytes, sl.stream) != cudaSuccess) {
        buf = nullptr;
        st = SAQ_ERR_OOM;
    }
    size_t off = 0;
    saq::EncodeJob jobs[saq::kMaxGroups];
    for (size_t i = 0; i < sl.groups.size(); ++i) {
        Group &g = sl.groups[i];
        const saq_model *m = s->models[(size_t)g.coll];
        uint8_t *b = static_cast<uint8_t *>(buf);
        const size_t r = (size_t)g.rows;
        g.X = reinterpret_cast<float *>(b + off);
        off += align256(sizeof(float) * r * (size_t)m->d);
        g.codes = b + off;
        off += align256(m->code_bytes * r);
        g.factors = reinterpret_cast<float *>(b + off);
        off += align256(sizeof(float) * r * (size_t)m->nf);
        g.scratch = b + off;
        off += m->dk > 0 ? align256(saq::encode_scratch_bytes(m, g.rows)) : 0;
        jobs[i] = saq::EncodeJob{m, g.X, g.rows, g.codes, g.factors, g.scratch};
    }
    sl.buf = static_cast<uint8_t *>(buf);
    if (st == SAQ_OK)
        for (const Piece &pc : sl.pieces) {
            const Group &g = sl.groups[(size_t)pc.group];
            const int d = s->models[(size_t)g.coll]->d;
            if (cudaMemcpyAsync(g.X + pc.off * d, pc.req->X + pc.r0 * d,
                                sizeof(float) * (size_t)pc.nr * d, cudaMemcpyHostToDevice,
                                sl.stream) != cudaSuccess)
                st = SAQ_ERR_CUDA;
        }
    if (st == SAQ_OK) {
        const saq_model *mg = jobs[0].m;
        if (sl.groups.size() == 1 && !saq::use_tc(mg)) {
            // a CUDA-core model (or one without kept dimensions) alone
            if (mg->dk == 0) st = saq::launch_rownorm2(mg, jobs[0].X, jobs[0].n, jobs[0].factors, mg->nf, sl.stream);
            else st = saq::encode_rows(mg, jobs[0].X, jobs[0].n, jobs[0].codes, jobs[0].factors,
                                       jobs[0].scratch, jobs[0].n, sl.stream, sl.err_dev);
        } else {
            st = saq::encode_grouped(jobs, (int)sl.groups.size(), sl.stream, sl.err_dev,
                                     sl.err_dev + 1);
        }
    }
    if (st == SAQ_OK && (cudaMemcpyAsync(sl.err_host, sl.err_dev, sizeof(int),
                                         cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                         cudaMemsetAsync(sl.err_dev, 0, sizeof(int), sl.stream) != cudaSuccess))
        st = SAQ_ERR_CUDA;
    sl.launch_status = st;  // applied to the requests at completion, under the lock
    for (const Piece &pc : sl.pieces) {
        if (st != SAQ_OK) break;
        const Group &g = sl.groups[(size_t)pc.group];
        const saq_model *m = s->models[(size_t)g.coll];
        const size_t cb = m->code_bytes;
        if (cb)
            cudaMemcpyAsync(pc.req->codes + pc.r0 * (int64_t)cb, g.codes + pc.off * (int64_t)cb,
                            cb * (size_t)pc.nr, cudaMemcpyDeviceToHost, sl.stream);
        cudaMemcpyAsync(pc.req->factors + pc.r0 * m->nf, g.factors + pc.off * m->nf,
                        sizeof(float) * (size_t)pc.nr * m->nf, cudaMemcpyDeviceToHost, sl.stream);
    }
    // the memory returns to the pool once the copies out are done
    if (buf) cudaFreeAsync(buf, sl.stream);
    auto *arg = new std::pair<saq_ingest *, Slot *>(s, &sl);
    if (cudaLaunchHostFunc(sl.stream, on_batch_done, arg) != cudaSuccess) {
        delete arg;
        sl.launch_status = SAQ_ERR_CUDA;
        cudaStreamSynchronize(sl.stream);
        return false;
    }
    return true;
}

void scheduler(saq_ingest *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap(s);
        for (Slot &sl : s->slots) {
            if (sl.busy) continue;
            if (!form_batch(s, sl)) break;  // nothing queued, or no budget left
            lk.unlock();
            const bool cb = launch_batch(s, sl);
            lk.lock();
            if (!cb) sl.finished = true;
        }
        bool busy = false, queued = false, ready = false;
        for (Slot &sl : s->slots) {
            busy |= sl.busy;
            ready |= sl.busy && sl.finished;
        }
        for (auto &q : s->queues) queued |= !q.empty();
        if (s->stopping && !busy && !queued) break;
        if (ready) continue;
        if (queued && !busy) {
            // nothing in flight and still nothing admitted: the budget cannot
            // hold the head request's next row (open() rules this out)
            for (auto &q : s->queues)
                if (!q.empty()) {
                    Request *r = q.front();
                    q.pop_front();
                    r->status = SAQ_ERR_OOM;
                    r->rows_done = r->n;
                    r->done = true;
                    r->t_done = Clock::now();
                    s->completed += 1;
                    break;
                }
            s->cv_done.notify_all();
            continue;
        }
        s->cv_sched.wait(lk);
    }
}

void free_slots(saq_ingest *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
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
    size_t one_batch = 0;
    int worst = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        if (!models[i]) return set_error(SAQ_ERR_INVALID, "collection %d is NULL", i);
        if (models[i]->device != dev)
            return set_error(SAQ_ERR_INVALID, "collection %d lives on another device", i);
        const size_t b = group_bytes(models[i], p->max_batch_rows);
        if (b > one_batch) {
            one_batch = b;
            worst = i;
        }
    }
    // admission needs room for at least one whole batch of any collection
    if (one_batch > p->hbm_budget_bytes)
        return set_error(SAQ_ERR_OOM,
                         "a batch of %d rows of collection %d (%zu bytes) would exceed the HBM "
                         "budget of %zu bytes", p->max_batch_rows, worst, one_batch,
                         p->hbm_budget_bytes);
    saq_ingest *s = new (std::nothrow) saq_ingest();
    if (!s) return set_error(SAQ_ERR_OOM, "host allocation failed");
    s->models.assign(models, models + n_models);
    s->p = *p;
    s->device = dev;
    s->queues.resize((size_t)n_models);
    s->slots.resize((size_t)p->slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&sl.err_dev, 4 * sizeof(int)) != cudaSuccess ||
            cudaMemset(sl.err_dev, 0, 4 * sizeof(int)) != cudaSuccess ||
            cudaHostAlloc(&sl.err_host, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            free_slots(s);
            delete s;
            return set_error(SAQ_ERR_OOM, "slot allocation failed");
        }
        *sl.err_host = 0;
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
    out->mixed_batches = s->mixed;
    out->deferred_batches = s->deferred;
    out->peak_bytes_in_flight = s->peak;
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
