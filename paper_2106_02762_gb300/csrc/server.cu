// Continuous-batching server (ttc_server_*).
//
// Graphs stay resident on the device.  ttc_serve_submit only queues a query;
// a worker thread packs the pending queries of each graph into one batched
// count launch (at most max_batch), runs launches for different graphs
// concurrently on a pool of streams ("slots"), and, as each launch's event
// completes, publishes its counts and the submit-to-completion latency for
// ttc_serve_poll.  Queries that arrive while a graph's batch is on the
// device wait for the next batch of that graph, which starts as soon as the
// previous one completes and a slot is free: new work is admitted while
// other work is still running.  One batch per graph is in flight at a time,
// so a graph's scratch memory is never shared by two launches.
//
// ttc_serve_load admits a new graph only if free device memory (minus the
// reserve) covers an estimate of its load footprint; otherwise it evicts the
// least recently used idle graphs (no queued or running queries) first.
//
// Every wait is bounded: the worker sleeps at most wait_limit_us (default
// 200 us) between polls, and ttc_serve_drain gives up after its timeout.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "graph.cuh"

namespace ttc {
void set_last_error(const std::string &m);
void normalise(const ttc_delta &d, int64_t out[3]);
uint64_t graph_device_bytes(const ttc_graph *g);
}  // namespace ttc

using namespace ttc;
using Clock = std::chrono::steady_clock;

namespace {

struct PendingQuery {
    uint64_t ticket;
    int64_t d[3];  // normalised
    Clock::time_point submit;
};

struct Result {
    bool done = false;
    ttc_status status = TTC_OK;
    uint64_t out[8] = {};
    double latency = 0;
};

struct Served {
    uint64_t id = 0;
    ttc_graph *g = nullptr;
    uint64_t last_use = 0;
    bool busy = false;  // a batch is on the device
    std::deque<PendingQuery> pending;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    Served *graph = nullptr;
    std::vector<PendingQuery> batch;
    uint32_t cap = 0;
    DevBuf<int64_t> dq;
    DevBuf<unsigned long long> acc;
    int64_t *h_dq = nullptr;
    unsigned long long *h_acc = nullptr;
};

}  // namespace

struct ttc_server {
    ttc_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable cv_done;  // wakes drainers
    std::thread worker;
    bool stop = false;
    bool paused = false;
    int device = 0;
    std::map<uint64_t, Served *> graphs;
    std::unordered_map<uint64_t, Result> results;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1, next_graph = 1, clock = 0;
    uint64_t queued = 0;
    ttc_server_stats st{};
    std::atomic<uint64_t> reserve{0};  // device bytes kept free by admission

    void run();
    bool complete_finished();
    bool launch_ready();
    void launch(Slot &slot, Served *sg);
};

namespace {

uint64_t footprint_estimate(uint64_t m) {
    // peak of the load: edge arrays, sort buffers, pair lists and triangle
    // records; generous so admission errs on the side of eviction
    return 96 * m + (64ull << 20);
}

}  // namespace

void ttc_server::launch(Slot &slot, Served *sg) {
    const uint32_t k = (uint32_t)std::min<size_t>(sg->pending.size(), opts.max_batch);
    slot.batch.assign(sg->pending.begin(), sg->pending.begin() + k);
    sg->pending.erase(sg->pending.begin(), sg->pending.begin() + k);
    queued -= k;
    if (slot.cap < k) {
        if (slot.h_dq) cudaFreeHost(slot.h_dq);
        if (slot.h_acc) cudaFreeHost(slot.h_acc);
        slot.h_dq = nullptr;
        slot.h_acc = nullptr;
        TTC_CUDA(cudaMallocHost(&slot.h_dq, 3 * (size_t)k * 8));
        TTC_CUDA(cudaMallocHost(&slot.h_acc, (8 * (size_t)k + 1) * 8));
        slot.dq.alloc(3 * (size_t)k, slot.stream);
        slot.acc.alloc(8 * (size_t)k + 1, slot.stream);
        slot.cap = k;
    }
    for (uint32_t i = 0; i < k; i++) memcpy(slot.h_dq + 3 * i, slot.batch[i].d, 24);
    cudaStream_t s = slot.stream;
    TTC_CUDA(cudaMemcpyAsync(slot.dq.get(), slot.h_dq, 3 * (size_t)k * 8, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemsetAsync(slot.acc.get(), 0, (8 * (size_t)k + 1) * 8, s));
    count_queue(sg->g, slot.dq.get(), k, slot.acc.get(), s);
    TTC_CUDA(cudaMemcpyAsync(slot.h_acc, slot.acc.get(), (8 * (size_t)k + 1) * 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaEventRecord(slot.done, s));
    slot.busy = true;
    slot.graph = sg;
    sg->busy = true;
    sg->last_use = ++clock;
    st.launches++;
}

bool ttc_server::complete_finished() {
    bool any = false;
    for (auto &slot : slots) {
        if (!slot.busy) continue;
        const cudaError_t e = cudaEventQuery(slot.done);
        if (e == cudaErrorNotReady) continue;
        const auto now = Clock::now();
        const uint32_t k = (uint32_t)slot.batch.size();
        const unsigned long long fl = e == cudaSuccess ? slot.h_acc[8 * (size_t)k] : 0ull;
        for (uint32_t i = 0; i < k; i++) {
            Result &r = results[slot.batch[i].ticket];
            r.done = true;
            r.status = e != cudaSuccess ? TTC_ERR_CUDA : (fl & 2ull) ? TTC_ERR_TIMEOUT : fl ? TTC_ERR_OVERFLOW : TTC_OK;
            if (e == cudaSuccess) memcpy(r.out, slot.h_acc + 8 * (size_t)i, 64);
            r.latency = std::chrono::duration<double>(now - slot.batch[i].submit).count();
        }
        if (e != cudaSuccess) cudaGetLastError();
        st.completed += k;
        slot.graph->busy = false;
        slot.busy = false;
        slot.graph = nullptr;
        slot.batch.clear();
        any = true;
    }
    return any;
}

bool ttc_server::launch_ready() {
    bool any = false;
    // oldest waiting query first across graphs
    std::vector<Served *> ready;
    for (auto &kv : graphs)
        if (!kv.second->busy && !kv.second->pending.empty()) ready.push_back(kv.second);
    std::sort(ready.begin(), ready.end(),
              [](Served *a, Served *b) { return a->pending.front().submit < b->pending.front().submit; });
    for (Served *sg : ready) {
        Slot *free_slot = nullptr;
        for (auto &slot : slots)
            if (!slot.busy) {
                free_slot = &slot;
                break;
            }
        if (!free_slot) break;
        try {
            launch(*free_slot, sg);
        } catch (const Failure &f) {
            // the batch's queries fail with the launch's status
            for (auto &q : free_slot->batch) {
                Result &r = results[q.ticket];
                r.done = true;
                r.status = f.status;
            }
            st.completed += free_slot->batch.size();
            free_slot->batch.clear();
            free_slot->busy = false;
            sg->busy = false;
        }
        any = true;
    }
    return any;
}

void ttc_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        const bool a = complete_finished();
        const bool b = paused ? false : launch_ready();
        if (a) cv_done.notify_all();
        if (!a && !b) cv.wait_for(lk, std::chrono::microseconds(opts.wait_limit_us));
    }
}

extern "C" {

ttc_server *ttc_server_create(const ttc_server_opts *o) {
    ttc_server *s = nullptr;
    try {
        s = new ttc_server();
        if (o) s->opts = *o;
        s->reserve.store(s->opts.hbm_reserve_bytes);
        if (!s->opts.max_batch) s->opts.max_batch = 256;
        if (!s->opts.max_queue) s->opts.max_queue = 65536;
        if (!s->opts.streams) s->opts.streams = 4;
        if (!s->opts.wait_limit_us) s->opts.wait_limit_us = 200;
        TTC_CUDA(cudaGetDevice(&s->device));
        s->slots.resize(s->opts.streams);
        for (auto &slot : s->slots) {
            TTC_CUDA(cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking));
            TTC_CUDA(cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming));
        }
        s->worker = std::thread([s] { s->run(); });
        return s;
    } catch (const Failure &f) {
        set_last_error(f.message);
    } catch (...) {
        set_last_error("server creation failed");
    }
    if (s) ttc_server_destroy(s);
    return nullptr;
}

void ttc_server_destroy(ttc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &slot : s->slots) {
        if (slot.stream) cudaStreamSynchronize(slot.stream);
        slot.dq.reset();
        slot.acc.reset();
        if (slot.h_dq) cudaFreeHost(slot.h_dq);
        if (slot.h_acc) cudaFreeHost(slot.h_acc);
        if (slot.done) cudaEventDestroy(slot.done);
        if (slot.stream) cudaStreamDestroy(slot.stream);
    }
    for (auto &kv : s->graphs) {
        ttc_free(kv.second->g);
        delete kv.second;
    }
    delete s;
}

ttc_status ttc_serve_load(ttc_server *s, const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                          uint64_t *graph_id) {
    if (!s || !graph_id || (m && (!src || !dst || !t))) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    try {
        TTC_CUDA(cudaSetDevice(s->device));
        const uint64_t need = footprint_estimate(m);
        // evict least recently used idle graphs until the estimate fits;
        // evict nothing when even evicting every idle graph would not do
        for (bool first = true;; first = false) {
            size_t free_b = 0, total_b = 0;
            TTC_CUDA(cudaMemGetInfo(&free_b, &total_b));
            free_b += pool_cached_bytes();  // freed blocks the library keeps for reuse
            const uint64_t reserve = s->reserve.load();
            const uint64_t avail = free_b > reserve ? free_b - reserve : 0;
            if (avail >= need) break;
            Served *victim = nullptr;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                uint64_t idle_bytes = 0;
                for (auto &kv : s->graphs) {
                    Served *c = kv.second;
                    if (c->busy || !c->pending.empty()) continue;
                    idle_bytes += graph_device_bytes(c->g);
                    if (!victim || c->last_use < victim->last_use) victim = c;
                }
                if (first && avail + idle_bytes < need) victim = nullptr;
                if (victim) {
                    s->graphs.erase(victim->id);
                    s->st.evictions++;
                }
            }
            if (!victim) fail(TTC_ERR_NOMEM, "not enough free device memory to admit %llu edges",
                              (unsigned long long)m);
            ttc_free(victim->g);
            delete victim;
        }
        ttc_graph *g = nullptr;
        const ttc_status rc = ttc_load_ex(src, dst, t, m, nullptr, &g);
        if (rc != TTC_OK) return rc;
        auto *sg = new Served();
        sg->g = g;
        std::lock_guard<std::mutex> lk(s->mu);
        sg->id = s->next_graph++;
        sg->last_use = ++s->clock;
        s->graphs[sg->id] = sg;
        s->st.admissions++;
        *graph_id = sg->id;
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    } catch (...) {
        set_last_error("unexpected internal failure");
        return TTC_ERR_INTERNAL;
    }
}

ttc_status ttc_serve_submit(ttc_server *s, uint64_t graph_id, const ttc_delta *d, uint64_t *ticket) {
    if (!s || !d || !ticket) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    PendingQuery q;
    try {
        normalise(*d, q.d);
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->graphs.find(graph_id);
        if (it == s->graphs.end()) {
            set_last_error("unknown or evicted graph id");
            return TTC_ERR_NOT_FOUND;
        }
        if (s->queued >= s->opts.max_queue) {
            set_last_error("server queue is full");
            return TTC_ERR_BUSY;
        }
        q.ticket = s->next_ticket++;
        q.submit = Clock::now();
        it->second->pending.push_back(q);
        it->second->last_use = ++s->clock;
        s->results[q.ticket] = Result{};
        s->queued++;
        s->st.submitted++;
        s->st.queue_depth_max = std::max<uint64_t>(s->st.queue_depth_max, s->queued);
        *ticket = q.ticket;
    }
    s->cv.notify_one();
    return TTC_OK;
}

ttc_status ttc_serve_poll(ttc_server *s, uint64_t ticket, uint64_t out[TTC_NUM_TYPES], double *latency_s) {
    if (!s || !out) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        set_last_error("unknown or already collected ticket");
        return TTC_ERR_NOT_FOUND;
    }
    if (!it->second.done) return TTC_PENDING;
    const Result r = it->second;
    s->results.erase(it);
    if (r.status != TTC_OK) {
        set_last_error(r.status == TTC_ERR_OVERFLOW ? "a count exceeds 2^64 - 1" : "the query's launch failed");
        return r.status;
    }
    memcpy(out, r.out, 64);
    if (latency_s) *latency_s = r.latency;
    return TTC_OK;
}

ttc_status ttc_serve_pause(ttc_server *s, int paused) {
    if (!s) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv.notify_all();
    return TTC_OK;
}

ttc_status ttc_serve_set_reserve(ttc_server *s, uint64_t hbm_reserve_bytes) {
    if (!s) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    s->reserve.store(hbm_reserve_bytes);
    return TTC_OK;
}

ttc_status ttc_serve_drain(ttc_server *s, double timeout_s) {
    if (!s) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                          timeout_s > 0 ? timeout_s : 0.0));
    while (s->st.completed < s->st.submitted) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && s->st.completed < s->st.submitted) {
            set_last_error("drain timed out");
            return TTC_ERR_TIMEOUT;
        }
    }
    return TTC_OK;
}

ttc_status ttc_server_info(ttc_server *s, ttc_server_stats *st) {
    if (!s || !st) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->graphs_resident = s->graphs.size();
    return TTC_OK;
}

}  // extern "C"
