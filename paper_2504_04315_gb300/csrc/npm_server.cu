// npm_server.cu -- continuous-batching request loop over one npm_handle
// (the batched per-bounce inference and interleaved training of Sec. 5.2).
//
// Callers submit query requests (guided sampling) and training requests from
// any host thread, with HOST arrays. A worker thread admits requests in
// arrival order as soon as space in a device staging pool allows (admission
// by memory), copies their inputs in, and serves every admitted query request
// with ONE launch of the fused forward kernel over a segment table; results
// are copied back and the request completes from a stream callback. Batches
// alternate between two streams so that a new batch starts while the previous
// one drains. A training request is ordered after every earlier query batch
// and before every later one (events), so queries see the weights of the
// training steps submitted before them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <algorithm>
#include <string.h>

#include "npm_handle.h"
#include "npm_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

// Rows of the staging pool (each row holds pool_queries floats).
enum { R_POS = 0, R_AUX = 3, R_U = 10, R_DIR = 14, R_PDF = 17, R_ROWS = 18 };

struct Request {
    uint64_t id;
    bool train;
    int64_t n, ld;
    const float* pos;
    const float* aux;
    const float* u;    // query: u [3/4][ld]; train: dir [3][ld]
    const float* rad;  // train: radiance [n]
    const float* spdf; // train: sample_pdf [n]
    float ufrac;
    float* dir_out;
    float* pdf_out;
    int64_t off = -1;  // pool offset once admitted
    Clock::time_point t_submit;
    double latency_ms = 0.0;
    bool done = false;
    npm_status status = NPM_OK;
};

struct Batch {
    struct npm_server* srv;
    std::vector<Request*> reqs;
};

}  // namespace

struct npm_server {
    npm_handle* h = nullptr;
    int64_t P = 0;  // pool capacity (queries)
    float* pool = nullptr;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t last_train = nullptr;  // completion of the latest training batch
    std::vector<cudaEvent_t> query_events;  // query batches launched since that training batch
    std::vector<cudaEvent_t> free_events;
    int next_stream = 0;
    bool have_train = false;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> all;
    std::map<int64_t, int64_t> free_list;  // offset -> length
    uint64_t next_id = 1;
    bool stop = false;
    bool hold = false;
    int inflight = 0;
    std::thread worker;

    // statistics
    int64_t batches = 0, requests_done = 0, queries_done = 0, train_done = 0;
    int max_per_batch = 0;
    int64_t pool_used = 0, pool_peak = 0;
    std::vector<double> latencies;
};

namespace {

// First-fit allocation of n contiguous pool queries; -1 if none.
int64_t pool_alloc(npm_server* s, int64_t n) {
    for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
        if (it->second >= n) {
            const int64_t off = it->first, len = it->second;
            s->free_list.erase(it);
            if (len > n) s->free_list[off + n] = len - n;
            s->pool_used += n;
            s->pool_peak = std::max(s->pool_peak, s->pool_used);
            return off;
        }
    }
    return -1;
}

void pool_free(npm_server* s, int64_t off, int64_t n) {
    s->pool_used -= n;
    auto it = s->free_list.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != s->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_list.erase(nx);
    }
    if (it != s->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_list.erase(it);
        }
    }
}

float* row(npm_server* s, int r, int64_t off) { return s->pool + (int64_t)r * s->P + off; }

// Stream callback: the batch's copies back to the host are complete.
void CUDART_CB on_batch_done(void* p) {
    Batch* b = static_cast<Batch*>(p);
    npm_server* s = b->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = Clock::now();
        for (Request* r : b->reqs) {
            r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
            r->done = true;
            pool_free(s, r->off, r->n);
            s->latencies.push_back(r->latency_ms);
            s->requests_done += 1;
            if (r->train)
                s->train_done += 1;
            else
                s->queries_done += r->n;
        }
        s->inflight -= 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    delete b;
}

cudaEvent_t take_event(npm_server* s) {
    if (!s->free_events.empty()) {
        cudaEvent_t e = s->free_events.back();
        s->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// rows x n block between [rows][ld] layouts: one strided copy (the worker
// thread's API calls per request are what a busy server pays for).
void copy_rows(float* dst, int64_t dst_ld, const float* src, int64_t src_ld, int rows, int64_t n,
               cudaMemcpyKind kind, cudaStream_t st) {
    if (rows == 1)
        cudaMemcpyAsync(dst, src, (size_t)n * sizeof(float), kind, st);
    else
        cudaMemcpy2DAsync(dst, (size_t)dst_ld * sizeof(float), src, (size_t)src_ld * sizeof(float),
                          (size_t)n * sizeof(float), rows, kind, st);
}

// Launches one batch (called by the worker without the lock held).
void launch_batch(npm_server* s, Batch* b) {
    npm_handle* h = s->h;
    const bool product = h->cfg.mode == NPM_PRODUCT;
    const bool train = b->reqs.size() == 1 && b->reqs[0]->train;
    cudaStream_t st = s->st[s->next_stream];
    s->next_stream ^= 1;
    if (train) {
        // After every query batch launched since the last training step.
        for (cudaEvent_t e : s->query_events) {
            cudaStreamWaitEvent(st, e, 0);
            s->free_events.push_back(e);
        }
        s->query_events.clear();
        if (s->have_train) cudaStreamWaitEvent(st, s->last_train, 0);
        Request* r = b->reqs[0];
        copy_rows(row(s, R_POS, r->off), s->P, r->pos, r->ld, 3, r->n, cudaMemcpyHostToDevice, st);
        if (product)
            copy_rows(row(s, R_AUX, r->off), s->P, r->aux, r->ld, 7, r->n, cudaMemcpyHostToDevice, st);
        copy_rows(row(s, R_U, r->off), s->P, r->u, r->ld, 3, r->n, cudaMemcpyHostToDevice, st);
        copy_rows(row(s, R_DIR, r->off), s->P, r->rad, r->n, 1, r->n, cudaMemcpyHostToDevice, st);
        copy_rows(row(s, R_PDF, r->off), s->P, r->spdf, r->n, 1, r->n, cudaMemcpyHostToDevice, st);
        r->status = npm_train_step(h, r->n, row(s, R_POS, r->off), product ? row(s, R_AUX, r->off) : nullptr,
                                   row(s, R_U, r->off), row(s, R_DIR, r->off), row(s, R_PDF, r->off),
                                   s->P, nullptr, st);
        cudaEventRecord(s->last_train, st);
        s->have_train = true;
    } else {
        if (s->have_train) cudaStreamWaitEvent(st, s->last_train, 0);
        npm::QueryBatch qb;
        memset(&qb, 0, sizeof(qb));
        qb.nseg = (int)b->reqs.size();
        qb.sample = 1;
        int64_t max_n = 0;
        for (int i = 0; i < qb.nseg; ++i) {
            Request* r = b->reqs[i];
            const int urows = r->ufrac > 0.0f ? 4 : 3;
            copy_rows(row(s, R_POS, r->off), s->P, r->pos, r->ld, 3, r->n, cudaMemcpyHostToDevice, st);
            if (product)
                copy_rows(row(s, R_AUX, r->off), s->P, r->aux, r->ld, 7, r->n, cudaMemcpyHostToDevice, st);
            copy_rows(row(s, R_U, r->off), s->P, r->u, r->ld, urows, r->n, cudaMemcpyHostToDevice, st);
            npm::QuerySeg& q = qb.seg[i];
            q.n = r->n;
            q.ld = s->P;
            q.pos = row(s, R_POS, r->off);
            q.aux = product ? row(s, R_AUX, r->off) : nullptr;
            q.uin = row(s, R_U, r->off);
            q.dir = row(s, R_DIR, r->off);
            q.pdf = row(s, R_PDF, r->off);
            q.mix = nullptr;
            q.ufrac = r->ufrac;
            max_n = std::max(max_n, r->n);
        }
        cudaError_t e = h->tc ? npm::tc_query_batch(h, qb, max_n, st)
                              : npm::launch_forward_fp32_batch(h->dc, inf_params(h), inf_wfwd(h), qb, max_n, st, status_word(h), h->wait_limit);
        for (Request* r : b->reqs) {
            r->status = e == cudaSuccess ? NPM_OK : NPM_ERR_CUDA;
            copy_rows(r->dir_out, r->ld, row(s, R_DIR, r->off), s->P, 3, r->n, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(r->pdf_out, row(s, R_PDF, r->off), (size_t)r->n * sizeof(float),
                            cudaMemcpyDeviceToHost, st);
        }
        // Events of query batches that have already finished need no wait.
        for (size_t i = 0; i < s->query_events.size();) {
            if (cudaEventQuery(s->query_events[i]) == cudaSuccess) {
                s->free_events.push_back(s->query_events[i]);
                s->query_events[i] = s->query_events.back();
                s->query_events.pop_back();
            } else {
                ++i;
            }
        }
        cudaGetLastError();
        cudaEvent_t ev = take_event(s);
        cudaEventRecord(ev, st);
        s->query_events.push_back(ev);
    }
    cudaLaunchHostFunc(st, on_batch_done, b);
}

void worker_loop(npm_server* s) {
    cudaSetDevice(s->h->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [s] { return s->stop || (!s->hold && !s->pending.empty()); });
        if (s->pending.empty()) {
            if (s->stop) break;
            continue;
        }
        // Admit in arrival order while memory allows. A training request
        // forms a batch of its own.
        Batch* b = new Batch();
        b->srv = s;
        while (!s->pending.empty() && (int)b->reqs.size() < npm::kMaxSegs) {
            Request* r = s->pending.front();
            if (r->train && !b->reqs.empty()) break;
            const int64_t off = pool_alloc(s, r->n);
            if (off < 0) break;
            r->off = off;
            s->pending.pop_front();
            b->reqs.push_back(r);
            if (r->train) break;
        }
        if (b->reqs.empty()) {
            delete b;
            // Nothing fits until a running batch frees pool space; its
            // completion callback notifies cv_work (it needs the lock, so the
            // notification cannot be missed between the check and the wait).
            s->cv_work.wait(lk);
            continue;
        }
        s->batches += 1;
        s->max_per_batch = std::max(s->max_per_batch, (int)b->reqs.size());
        s->inflight += 1;
        lk.unlock();
        launch_batch(s, b);
        lk.lock();
    }
}

npm_status submit(npm_server* s, Request* r, uint64_t* ticket) {
    if (r->n > s->P || r->n > s->h->cfg.max_batch) {
        delete r;
        return npm::set_error(NPM_ERR_CAPACITY,
                              "request larger than the staging pool or the handle's max_batch");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return npm::set_error(NPM_ERR_INVALID_ARG, "server is shutting down");
        }
        r->id = s->next_id++;
        r->t_submit = Clock::now();
        s->all[r->id] = r;
        s->pending.push_back(r);
        *ticket = r->id;
    }
    s->cv_work.notify_all();
    return NPM_OK;
}

}  // namespace

extern "C" {

npm_status npm_server_create(npm_handle* h, int64_t pool_queries, npm_server** out) {
    npm::CallRange range("npm_server_create");
    if (!h || !out || pool_queries < 1) return npm::set_error(NPM_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    npm_server* s = new npm_server();
    s->h = h;
    s->P = pool_queries;
    if (cudaMalloc(&s->pool, sizeof(float) * (size_t)R_ROWS * pool_queries) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return npm::set_error(NPM_ERR_OOM, "cannot allocate the staging pool");
    }
    bool ok = true;
    for (int i = 0; i < 2; ++i) ok = ok && cudaStreamCreateWithFlags(&s->st[i], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->last_train, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        const char* msg = cudaGetErrorString(cudaGetLastError());
        for (int i = 0; i < 2; ++i)
            if (s->st[i]) cudaStreamDestroy(s->st[i]);
        if (s->last_train) cudaEventDestroy(s->last_train);
        cudaFree(s->pool);
        delete s;
        return npm::set_error(NPM_ERR_CUDA, msg);
    }
    s->free_list[0] = pool_queries;
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return NPM_OK;
}

npm_status npm_server_submit_query(npm_server* s, int64_t n, const float* pos, const float* aux,
                                   const float* u, int64_t ld, float uniform_frac, float* dir_out,
                                   float* pdf_out, uint64_t* ticket) {
    npm::CallRange range("npm_server_submit_query");
    if (!s || !ticket || n < 1 || ld < n || !pos || !u || !dir_out || !pdf_out ||
        (s->h->cfg.mode == NPM_PRODUCT && !aux) || !(uniform_frac >= 0.0f && uniform_frac <= 1.0f))
        return npm::set_error(NPM_ERR_INVALID_ARG, "bad query request");
    Request* r = new Request();
    r->train = false;
    r->n = n;
    r->ld = ld;
    r->pos = pos;
    r->aux = aux;
    r->u = u;
    r->rad = r->spdf = nullptr;
    r->ufrac = uniform_frac;
    r->dir_out = dir_out;
    r->pdf_out = pdf_out;
    return submit(s, r, ticket);
}

npm_status npm_server_submit_train(npm_server* s, int64_t n, const float* pos, const float* aux,
                                   const float* dir, const float* radiance, const float* sample_pdf,
                                   int64_t ld, uint64_t* ticket) {
    npm::CallRange range("npm_server_submit_train");
    if (!s || !ticket || n < 1 || ld < n || !pos || !dir || !radiance || !sample_pdf ||
        (s->h->cfg.mode == NPM_PRODUCT && !aux))
        return npm::set_error(NPM_ERR_INVALID_ARG, "bad training request");
    Request* r = new Request();
    r->train = true;
    r->n = n;
    r->ld = ld;
    r->pos = pos;
    r->aux = aux;
    r->u = dir;
    r->rad = radiance;
    r->spdf = sample_pdf;
    r->ufrac = 0.0f;
    r->dir_out = nullptr;
    r->pdf_out = nullptr;
    return submit(s, r, ticket);
}

npm_status npm_server_wait(npm_server* s, uint64_t ticket, double* latency_ms) {
    npm::CallRange range("npm_server_wait");
    if (!s) return npm::set_error(NPM_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return npm::set_error(NPM_ERR_INVALID_ARG, "unknown ticket");
    Request* r = it->second;
    s->cv_done.wait(lk, [r] { return r->done; });
    if (latency_ms) *latency_ms = r->latency_ms;
    const npm_status st = r->status;
    s->all.erase(it);
    delete r;
    if (st != NPM_OK) return npm::set_error(st, "request failed");
    return NPM_OK;
}

npm_status npm_server_hold(npm_server* s, int hold) {
    if (!s) return npm::set_error(NPM_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->hold = hold != 0;
    }
    s->cv_work.notify_all();
    return NPM_OK;
}

npm_status npm_server_get_stats(npm_server* s, npm_server_stats* out) {
    if (!s || !out) return npm::set_error(NPM_ERR_INVALID_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->batches = s->batches;
    out->requests_done = s->requests_done;
    out->queries_done = s->queries_done;
    out->train_done = s->train_done;
    out->max_requests_per_batch = s->max_per_batch;
    out->pool_queries = s->P;
    out->pool_peak_used = s->pool_peak;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        out->latency_p50_ms = v[v.size() / 2];
        out->latency_p99_ms = v[std::min(v.size() - 1, (size_t)(0.99 * (double)v.size()))];
    }
    return NPM_OK;
}

npm_status npm_server_destroy(npm_server* s) {
    npm::CallRange range("npm_server_destroy");
    if (!s) return NPM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->hold = false;
    }
    s->cv_work.notify_all();
    s->worker.join();
    for (int i = 0; i < 2; ++i) cudaStreamSynchronize(s->st[i]);
    {
        // Callbacks of the last batches may still be running.
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [s] { return s->inflight == 0; });
    }
    for (auto& kv : s->all) delete kv.second;
    for (cudaEvent_t e : s->query_events) cudaEventDestroy(e);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    cudaEventDestroy(s->last_train);
    for (int i = 0; i < 2; ++i) cudaStreamDestroy(s->st[i]);
    cudaFree(s->pool);
    delete s;
    return NPM_OK;
}

}  // extern "C"
