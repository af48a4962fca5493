// Serving loop: continuous batching of new-item what-if queries over resident users.
//
// Each request is Definition 2 for new items (counts[j] = #{u : u.Q_j > tau_u}, the new
// item losing ties), computed by the same counting pass as rkm_query_new_items.  The paper
// has no serving loop; this file is the request queue around that pass:
//  * submit appends the request to a FIFO queue (host buffers borrowed until it finishes);
//  * every slot (a worker thread with its own stream and workspace) that becomes free takes
//    the oldest waiting requests, as many as fit max_batch_items and the free part of the
//    device arena (serve_sched.h), stages their rows through its pinned buffer to the arena,
//    runs one counting pass over the users for the whole batch, copies the counts back and
//    completes the requests;
//  * several slots keep several batches on the device at once, so the copies and host work
//    of one batch overlap the kernels of another, and requests that arrive while batches run
//    are admitted as soon as a slot and arena memory free up.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rkm.h"
#include "internal.h"
#include "serve_sched.h"

namespace {

using rkm::serve::Arena;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    const float* Q;
    int64_t q, ldq;
    int32_t* counts;
    double t_submit = 0, t_admit = 0, t_done = 0;
    rkm_status status = RKM_OK;
    std::string error;
    bool done = false;
};

struct Slot {
    rkm_ctx* work = nullptr;
    cudaStream_t stream = nullptr;
    float* h_rows = nullptr;    // pinned staging of a batch's candidate rows
    int32_t* h_counts = nullptr;  // pinned staging of its counts
    std::thread thread;
};

}  // namespace

struct rkm_server {
    rkm_ctx* owner = nullptr;
    rkm_serve_opts opts{};
    int device = 0, d = 0;
    int64_t n = 0;
    char* arena_base = nullptr;
    Arena arena;
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv_work;  // a request arrived, memory was released, or stopping
    std::condition_variable cv_done;  // a request finished
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, Request*> tickets;
    uint64_t next_ticket = 1;
    int running = 0;  // batches admitted and not finished
    bool stopping = false;

    // statistics since the last reset (under mu)
    std::vector<double> latency;
    double queue_sum = 0, t_first = -1, t_last = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, items = 0, batches = 0;
    int max_in_flight = 0;
    unsigned long long launches0 = 0;

    void worker(Slot& sl);
    rkm_status run_batch(Slot& sl, const std::vector<Request*>& batch, int64_t items_total, size_t off);
};

namespace {

rkm_status fail(rkm_status s, const std::string& msg) { return rkm::fail_with(s, msg.c_str()); }

std::string cuda_msg(const char* what, cudaError_t e) { return std::string(what) + ": " + cudaGetErrorString(e); }

}  // namespace

// One batch on slot `sl`: stage the rows, count, return the counts.  Runs without the lock.
rkm_status rkm_server::run_batch(Slot& sl, const std::vector<Request*>& batch, int64_t items_total, size_t off) {
    float* d_rows = reinterpret_cast<float*>(arena_base + off);
    int32_t* d_counts = reinterpret_cast<int32_t*>(arena_base + off +
                                                   rkm::serve::round_granule((size_t)items_total * d * sizeof(float)));
    int64_t row = 0;
    for (const Request* r : batch) {
        float* dst = sl.h_rows + row * d;
        if (r->ldq == d) {
            std::memcpy(dst, r->Q, (size_t)r->q * d * sizeof(float));
        } else {
            for (int64_t j = 0; j < r->q; ++j) std::memcpy(dst + j * d, r->Q + j * r->ldq, (size_t)d * sizeof(float));
        }
        row += r->q;
    }
    cudaError_t e = cudaMemcpyAsync(d_rows, sl.h_rows, (size_t)items_total * d * sizeof(float),
                                    cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return fail(RKM_ECUDA, cuda_msg("candidate upload", e));
    const rkm_status st = rkm::query_resident(sl.work, owner, d_rows, items_total, d, d_counts, sl.stream);
    if (st != RKM_OK) return st;
    e = cudaMemcpyAsync(sl.h_counts, d_counts, (size_t)items_total * sizeof(int32_t), cudaMemcpyDeviceToHost,
                        sl.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.stream);
    if (e != cudaSuccess) return fail(RKM_ECUDA, cuda_msg("count download", e));
    row = 0;
    for (Request* r : batch) {
        std::memcpy(r->counts, sl.h_counts + row, (size_t)r->q * sizeof(int32_t));
        row += r->q;
    }
    return RKM_OK;
}

void rkm_server::worker(Slot& sl) {
    cudaSetDevice(device);
    std::vector<Request*> batch;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        size_t off = 0;
        int64_t total = 0;
        int count = 0;
        for (;;) {
            if (!waiting.empty()) {
                count = rkm::serve::take_batch(
                    waiting.size(), [&](size_t j) { return waiting[j]->q; }, opts.max_batch_items, d, arena, &off,
                    &total);
                if (count > 0) break;
            } else if (stopping) {
                return;
            }
            cv_work.wait(lk);
        }
        batch.assign(waiting.begin(), waiting.begin() + count);
        waiting.erase(waiting.begin(), waiting.begin() + count);
        const double t_admit = now_ms();
        for (Request* r : batch) r->t_admit = t_admit;
        ++running;
        max_in_flight = std::max(max_in_flight, running);
        lk.unlock();

        const rkm_status st = run_batch(sl, batch, total, off);
        const std::string msg = st == RKM_OK ? std::string() : std::string(rkm_last_error());
        const double t_done = now_ms();

        lk.lock();
        arena.release(off, rkm::serve::batch_bytes(total, d));
        --running;
        ++batches;
        for (Request* r : batch) {
            r->status = st;
            r->error = msg;
            r->t_done = t_done;
            r->done = true;
            latency.push_back(t_done - r->t_submit);
            queue_sum += r->t_admit - r->t_submit;
            ++completed;
            if (st != RKM_OK) ++failed;
            items += (uint64_t)r->q;
        }
        t_last = std::max(t_last, t_done);
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

void rkm_serve_default_opts(rkm_serve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->slots = 2;
    o->max_batch_items = 8192;
    o->memory_bytes = 64ll << 20;
    o->max_pending = 1 << 20;
}

void rkm_serve_destroy(rkm_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    for (Slot& sl : srv->slots)
        if (sl.thread.joinable()) sl.thread.join();
    cudaSetDevice(srv->device);
    for (Slot& sl : srv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.work) rkm_destroy(sl.work);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_rows) cudaFreeHost(sl.h_rows);
        if (sl.h_counts) cudaFreeHost(sl.h_counts);
    }
    if (srv->arena_base) cudaFree(srv->arena_base);
    for (auto& t : srv->tickets) delete t.second;
    if (srv->owner) rkm::attach_server(srv->owner, -1);
    delete srv;
}

rkm_status rkm_serve_create(rkm_server** out, rkm_ctx* ctx, const rkm_serve_opts* opts) {
    if (!out || !ctx) return fail(RKM_EINVAL, "null argument");
    *out = nullptr;
    rkm_serve_opts o;
    rkm_serve_default_opts(&o);
    if (opts) o = *opts;
    if (o.slots < 1 || o.slots > 16) return fail(RKM_EINVAL, "slots must be in [1, 16]");
    if (o.max_batch_items < 1 || o.max_batch_items > (1 << 24))
        return fail(RKM_EINVAL, "max_batch_items must be in [1, 2^24]");
    if (o.max_pending < 1) return fail(RKM_EINVAL, "max_pending must be >= 1");
    int64_t n = 0;
    int d = 0, device = 0;
    if (!rkm::resident_shape(ctx, &n, &d, &device)) return fail(RKM_ESTATE, "rkm_serve_create before rkm_resident_set");
    if (o.memory_bytes < (int64_t)rkm::serve::batch_bytes(1, d))
        return fail(RKM_EINVAL, "memory_bytes cannot hold a single candidate");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(RKM_ECUDA, cuda_msg("cudaSetDevice", e));

    rkm_server* srv = new rkm_server();
    srv->owner = ctx;
    rkm::attach_server(ctx, +1);
    srv->opts = o;
    srv->device = device;
    srv->d = d;
    srv->n = n;
    srv->slots.resize(o.slots);
    auto bail = [&](rkm_status s, const std::string& msg) {
        rkm_serve_destroy(srv);
        return fail(s, msg);
    };
    e = cudaMalloc(&srv->arena_base, (size_t)o.memory_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        srv->arena_base = nullptr;
        return bail(RKM_ENOMEM, cuda_msg("serving arena", e));
    }
    srv->arena.reset((size_t)o.memory_bytes);
    // Each slot: workspace sized by a warm-up pass of max_batch_items zero candidates (so that
    // serving allocates nothing unless a band queue overflows), a stream and pinned staging.
    const int64_t B = o.max_batch_items;
    float* zeros = nullptr;
    int32_t* zcounts = nullptr;
    e = cudaMalloc(&zeros, (size_t)B * d * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&zcounts, (size_t)B * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(zeros, 0, (size_t)B * d * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (zeros) cudaFree(zeros);
        if (zcounts) cudaFree(zcounts);
        return bail(RKM_ENOMEM, cuda_msg("warm-up buffers", e));
    }
    rkm_status st = RKM_OK;
    std::string msg;
    for (Slot& sl : srv->slots) {
        sl.work = rkm::worker_context(ctx);
        if (!sl.work) {
            st = RKM_ENOMEM;
            msg = "slot context allocation failed";
            break;
        }
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_rows, (size_t)B * d * sizeof(float));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_counts, (size_t)B * sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = RKM_ENOMEM;
            msg = cuda_msg("slot stream or staging", e);
            break;
        }
        st = rkm::query_resident(sl.work, ctx, zeros, B, d, zcounts, sl.stream);
        if (st != RKM_OK) {
            msg = std::string("slot warm-up: ") + rkm_last_error();
            break;
        }
    }
    cudaFree(zeros);
    cudaFree(zcounts);
    if (st != RKM_OK) return bail(st, msg);
    srv->launches0 = rkm::launch_count();
    for (Slot& sl : srv->slots) sl.thread = std::thread([srv, &sl] { srv->worker(sl); });
    *out = srv;
    return RKM_OK;
}

rkm_status rkm_serve_submit(rkm_server* srv, const float* Q, int64_t q, int64_t ldq, int32_t* counts,
                            uint64_t* ticket) {
    if (!srv || !Q || !counts || !ticket) return fail(RKM_EINVAL, "null argument");
    if (q < 1 || q > srv->opts.max_batch_items)
        return fail(RKM_EINVAL, "q must be in [1, max_batch_items] (got " + std::to_string(q) + ")");
    if (ldq < srv->d) return fail(RKM_EINVAL, "ldq < d");
    if (rkm::serve::batch_bytes(q, srv->d) > srv->arena.size())
        return fail(RKM_EINVAL, "request needs more device memory than the serving arena holds");
    Request* r = new Request();
    r->Q = Q;
    r->q = q;
    r->ldq = ldq;
    r->counts = counts;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) {
            delete r;
            return fail(RKM_ESTATE, "the server is stopping");
        }
        if ((int64_t)srv->waiting.size() >= srv->opts.max_pending) {
            delete r;
            return fail(RKM_EBUSY, "request queue full");
        }
        r->t_submit = now_ms();
        if (srv->t_first < 0) srv->t_first = r->t_submit;
        *ticket = srv->next_ticket++;
        srv->tickets[*ticket] = r;
        srv->waiting.push_back(r);
        ++srv->submitted;
    }
    srv->cv_work.notify_one();
    return RKM_OK;
}

rkm_status rkm_serve_wait(rkm_server* srv, uint64_t ticket, double timeout_ms, double* latency_ms) {
    if (!srv) return fail(RKM_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return fail(RKM_EINVAL, "unknown ticket " + std::to_string(ticket));
    Request* r = it->second;
    auto finished = [r] { return r->done; };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, finished);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), finished)) {
        return fail(RKM_ETIMEOUT, "request not finished within the timeout");
    }
    srv->tickets.erase(it);
    lk.unlock();
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    const rkm_status st = r->status;
    const std::string msg = r->error;
    delete r;
    if (st != RKM_OK) return fail(st, msg);
    return RKM_OK;
}

rkm_status rkm_serve_drain(rkm_server* srv) {
    if (!srv) return fail(RKM_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_done.wait(lk, [srv] { return srv->waiting.empty() && srv->running == 0; });
    return RKM_OK;
}

rkm_status rkm_serve_get_stats(rkm_server* srv, rkm_serve_stats* out) {
    if (!srv || !out) return fail(RKM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    rkm_serve_stats s;
    std::memset(&s, 0, sizeof s);
    s.submitted = srv->submitted;
    s.completed = srv->completed;
    s.failed = srv->failed;
    s.items = srv->items;
    s.batches = srv->batches;
    s.mean_batch_items = srv->batches ? (double)srv->items / (double)srv->batches : 0.0;
    if (!srv->latency.empty()) {
        std::vector<double> v(srv->latency);
        std::sort(v.begin(), v.end());
        auto rank = [&](double p) {  // nearest rank: the smallest value with at least p of the samples at or below it
            size_t i = (size_t)std::ceil(p * (double)v.size());
            return v[std::min(v.size(), std::max<size_t>(i, 1)) - 1];
        };
        s.p50_ms = rank(0.50);
        s.p99_ms = rank(0.99);
        s.max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        s.mean_ms = sum / (double)v.size();
        s.mean_queue_ms = srv->queue_sum / (double)v.size();
    }
    if (srv->t_first >= 0 && srv->completed) {
        s.window_ms = srv->t_last - srv->t_first;
        if (s.window_ms > 0) {
            s.items_per_s = (double)srv->items / (s.window_ms * 1e-3);
            s.pairs_per_s = s.items_per_s * (double)srv->n;
        }
    }
    s.arena_peak_bytes = (int64_t)srv->arena.high_water();
    s.max_in_flight = srv->max_in_flight;
    s.slots = (int32_t)srv->slots.size();
    s.kernel_launches = rkm::launch_count() - srv->launches0;
    *out = s;
    return RKM_OK;
}

rkm_status rkm_serve_reset_stats(rkm_server* srv) {
    if (!srv) return fail(RKM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->latency.clear();
    srv->queue_sum = 0;
    srv->t_first = -1;
    srv->t_last = 0;
    srv->submitted = srv->completed = srv->failed = srv->items = srv->batches = 0;
    srv->max_in_flight = srv->running;
    srv->arena.reset_high_water();
    srv->launches0 = rkm::launch_count();
    return RKM_OK;
}

}  // extern "C"
