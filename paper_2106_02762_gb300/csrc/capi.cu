// C-ABI entry points (include/ttc.h): argument checks, handle lifetime,
// delta normalisation, and conversion of internal failures to ttc_status.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "graph.cuh"

namespace ttc {

namespace {
thread_local std::string g_last_error;
thread_local int t_prof_off = 0;
std::atomic<uint64_t> g_fail_after{0};
std::atomic<uint64_t> g_bytes{0};
std::atomic<uint64_t> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfOff::ProfOff() { t_prof_off++; }
ProfOff::~ProfOff() { t_prof_off--; }

void prof_reset(ttc_graph *g) {
    if (!t_prof_off) g->prof_used = 0;
}

// Every load phase and count kernel is also an NVTX range (named as in the
// profile), so a timeline tool shows the stages.
void prof_begin(ttc_graph *g, cudaStream_t s, const char *name) {
    nvtxRangePushA(name);
    if (!g->profiling || t_prof_off) return;
    if (g->prof_used == g->prof.size()) {
        ttc_graph::ProfEntry e{name, nullptr, nullptr};
        TTC_CUDA(cudaEventCreate(&e.start));
        TTC_CUDA(cudaEventCreate(&e.stop));
        g->prof.push_back(e);
    }
    g->prof[g->prof_used].name = name;
    TTC_CUDA(cudaEventRecord(g->prof[g->prof_used].start, s));
}

void prof_end(ttc_graph *g, cudaStream_t s) {
    nvtxRangePop();
    if (!g->profiling || t_prof_off) return;
    TTC_CUDA(cudaEventRecord(g->prof[g->prof_used].stop, s));
    g->prof_used++;
}

// Normalises k device delta-triples in place (see normalise()).
__global__ void normalise_kernel(int64_t *d, uint32_t k) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    const int64_t d13 = d[3 * q], d12 = min(d[3 * q + 1], d13), d23 = min(d[3 * q + 2], d13);
    d[3 * q] = min(d13, d12 + d23);
    d[3 * q + 1] = d12;
    d[3 * q + 2] = d23;
}

void fail(ttc_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    throw Failure{st, buf};
}

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    const ttc_status st = e == cudaErrorMemoryAllocation ? TTC_ERR_NOMEM : TTC_ERR_CUDA;
    fail(st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

cudaMemPool_t library_pool();

void *device_alloc(size_t bytes, cudaStream_t s) {
    uint64_t n = g_fail_after.load();
    while (n) {
        if (g_fail_after.compare_exchange_weak(n, n - 1)) {
            if (n == 1) fail(TTC_ERR_NOMEM, "device allocation of %zu bytes failed (injected)", bytes);
            break;
        }
    }
    void *p = nullptr;
    cudaMemPool_t pool = library_pool();
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    if (e != cudaSuccess) {
        // give cached blocks back to the device and try once more
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(TTC_ERR_NOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    g_bytes += bytes;
    return p;
}

// One stream-ordered memory pool per device for everything the library
// allocates.  Its release threshold is unbounded, so blocks freed by
// ttc_free or by a load's temporaries are kept mapped and reused by the next
// load instead of being unmapped at every stream synchronisation (the
// default pool's behaviour).  pool_cached_bytes() reports what it holds
// unused, which admission control counts as free.
cudaMemPool_t library_pool() {
    constexpr int MAXDEV = 64;
    static cudaMemPool_t pools[MAXDEV] = {};
    static std::mutex mu;
    int dev = 0;
    TTC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAXDEV) fail(TTC_ERR_INTERNAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        TTC_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t thr = UINT64_MAX;
        TTC_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        pools[dev] = p;
    }
    return pools[dev];
}

uint64_t pool_cached_bytes() {
    cudaMemPool_t p = library_pool();
    uint64_t reserved = 0, used = 0;
    TTC_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &reserved));
    TTC_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &used));
    return reserved > used ? reserved - used : 0;
}

void device_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

uint64_t device_bytes_in_use() { return g_bytes.load(); }

int sm_count() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> counts[MAXDEV] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAXDEV) dev = 0;
    int n = counts[dev].load(std::memory_order_relaxed);
    if (!n) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        counts[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

void ensure_smem(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::set<std::tuple<const void *, int, size_t>> done;
    int dev = 0;
    TTC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({fn, dev, bytes})) return;
    TTC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.insert({fn, dev, bytes});
}

void set_last_error(const std::string &m) { g_last_error = m; }

void check_count_flag(unsigned long long flag) {
    if (take_bounds_word()) fail(TTC_ERR_INTERNAL, "a count kernel read an index outside its array (index checks)");
    if (flag & 2ull) fail(TTC_ERR_TIMEOUT, "a bounded wait in a count kernel gave up (bulk copy not complete)");
    if (flag) fail(TTC_ERR_OVERFLOW, "a count exceeds 2^64 - 1");
}

// Normalised copy of a delta-triple (leaves every count unchanged):
//   d12 <- min(d12, d13), d23 <- min(d23, d13), d13 <- min(d13, d12 + d23).
void normalise(const ttc_delta &d, int64_t out[3]) {
    const int64_t LIM = int64_t(1) << 62;
    if (d.d13 < 0 || d.d12 < 0 || d.d23 < 0 || d.d13 > LIM || d.d12 > LIM || d.d23 > LIM)
        fail(TTC_ERR_RANGE, "delta components must lie in [0, 2^62]");
    const int64_t d12 = d.d12 < d.d13 ? d.d12 : d.d13;
    const int64_t d23 = d.d23 < d.d13 ? d.d23 : d.d13;
    const int64_t d13 = d.d13 < d12 + d23 ? d.d13 : d12 + d23;
    out[0] = d13; out[1] = d12; out[2] = d23;
}

}  // namespace ttc

using namespace ttc;

#define TTC_API_BEGIN try {
#define TTC_API_END                                    \
    }                                                  \
    catch (const Failure &f) {                         \
        set_last_error(f.message);                     \
        return f.status;                               \
    }                                                  \
    catch (const std::bad_alloc &) {                   \
        set_last_error("host allocation failed");      \
        return TTC_ERR_NOMEM;                          \
    }                                                  \
    catch (...) {                                      \
        set_last_error("unexpected internal failure"); \
        return TTC_ERR_INTERNAL;                       \
    }

namespace ttc {
void multi_forget(ttc_graph *g);
void count_multi(ttc_graph *const *gs, const ttc_delta *d, uint32_t G, uint64_t *out);

// Device bytes a resident graph holds.
uint64_t graph_device_bytes(const ttc_graph *g) {
    return g->key.bytes() + g->fwd.bytes() + g->poff.bytes() + g->pair_vtx.bytes() + g->tri.bytes() +
           g->shard_view.bytes() + g->shard_pre.bytes() + g->shard_eoff.bytes() +
           g->huge_eoff.bytes() + g->view.bytes() + g->prefix.bytes() + g->acc.bytes() +
           g->dq.bytes() + g->scratch.bytes() + g->s_items.bytes() + g->s_ocsr.bytes() + g->s_onbr.bytes() +
           g->s_osrc.bytes() + g->s_in_e.bytes() + g->s_out_off.bytes() + g->s_in_off.bytes();
}
}  // namespace ttc

namespace {

void graph_destroy(ttc_graph *g) {
    if (!g) return;
    multi_forget(g);
    cudaSetDevice(g->device);
    cudaStream_t s = g->stream;
    for (auto &e : g->prof) {
        cudaEventDestroy(e.start);
        cudaEventDestroy(e.stop);
    }
    g->key.reset(); g->fwd.reset(); g->poff.reset(); g->pair_vtx.reset(); g->tri.reset();
    g->huge_eoff.reset(); g->view.reset(); g->prefix.reset();
    g->acc.reset(); g->dq.reset(); g->scratch.reset();
    g->shard_view.reset(); g->shard_pre.reset(); g->shard_eoff.reset();
    g->s_items.reset(); g->s_ocsr.reset(); g->s_onbr.reset(); g->s_osrc.reset(); g->s_in_e.reset();
    g->s_out_off.reset(); g->s_in_off.reset();
    // every buffer is freed on the graph's stream, so before that stream goes
    if (s) cudaStreamSynchronize(s);
    if (g->side) {
        cudaStreamSynchronize(g->side);
        cudaStreamDestroy(g->side);
        cudaEventDestroy(g->side_fork);
        cudaEventDestroy(g->side_join);
    }
    if (g->own_stream && s) cudaStreamDestroy(s);
    delete g;
}

// Runs k normalised queries and copies the counts to out (host); nshards > 0:
// only shard `shard` of that many.
ttc_status run_queries(ttc_graph *g, const ttc_delta *d, uint32_t k, uint64_t *out, uint32_t shard = 0,
                       uint32_t nshards = 0) {
    std::vector<int64_t> hq(3 * (size_t)k);
    for (uint32_t q = 0; q < k; q++) normalise(d[q], &hq[3 * (size_t)q]);
    std::lock_guard<std::mutex> lock(g->mu);
    TTC_CUDA(cudaSetDevice(g->device));
    cudaStream_t s = g->stream;
    if (g->acc_cap < k) {
        g->acc.alloc(8 * (size_t)k + 1, s);
        g->dq.alloc(3 * (size_t)k, s);
        g->acc_cap = k;
    }
    TTC_CUDA(cudaMemcpyAsync(g->dq.get(), hq.data(), hq.size() * 8, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemsetAsync(g->acc.get(), 0, (8 * (size_t)k + 1) * 8, s));
    prof_reset(g);
    if (nshards) count_queue_shard(g, g->dq.get(), k, g->acc.get(), shard, nshards, s);
    else count_queue(g, g->dq.get(), k, g->acc.get(), s);
    std::vector<unsigned long long> h(8 * (size_t)k + 1);
    TTC_CUDA(cudaMemcpyAsync(h.data(), g->acc.get(), h.size() * 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    check_count_flag(h[8 * (size_t)k]);
    memcpy(out, h.data(), 8 * (size_t)k * 8);
    return TTC_OK;
}

}  // namespace

extern "C" {

const char *ttc_last_error(void) { return g_last_error.c_str(); }

#ifndef TTC_COUNT_HASH
#define TTC_COUNT_HASH "unknown"
#endif
const char *ttc_version(void) { return "ttc 0.1 (sm_103a) count:" TTC_COUNT_HASH; }

ttc_status ttc_release_cached(uint64_t *released) {
    try {
        cudaMemPool_t pool = library_pool();
        uint64_t before = 0, after = 0;
        TTC_CUDA(cudaDeviceSynchronize());
        TTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &before));
        TTC_CUDA(cudaMemPoolTrimTo(pool, 0));
        TTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &after));
        if (released) *released = before > after ? before - after : 0;
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    }
}

ttc_status ttc_memory_info(uint64_t *device_free, uint64_t *pool_reserved, uint64_t *pool_used) {
    try {
        cudaMemPool_t pool = library_pool();
        size_t free_b = 0, total_b = 0;
        uint64_t reserved = 0, used = 0;
        TTC_CUDA(cudaMemGetInfo(&free_b, &total_b));
        TTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
        TTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
        if (device_free) *device_free = free_b;
        if (pool_reserved) *pool_reserved = reserved;
        if (pool_used) *pool_used = used;
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    }
}

void ttc_debug_fail_alloc_after(uint64_t n) { g_fail_after.store(n); }

uint64_t ttc_debug_launch_count(void) { return g_launches.load(); }

ttc_status ttc_set_profiling(ttc_graph *g, int on) {
    if (!g) {
        set_last_error("NULL graph");
        return TTC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g->mu);
    g->profiling = on != 0;
    g->prof_used = 0;
    return TTC_OK;
}

uint32_t ttc_profile_read(ttc_graph *g, ttc_kernel_time *out, uint32_t cap) {
    if (!g || !out) return 0;
    std::lock_guard<std::mutex> lock(g->mu);
    uint32_t n = 0;
    for (size_t i = 0; i < g->prof_used && n < cap; i++) {
        float ms = 0.f;
        if (cudaEventSynchronize(g->prof[i].stop) != cudaSuccess ||
            cudaEventElapsedTime(&ms, g->prof[i].start, g->prof[i].stop) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        snprintf(out[n].name, sizeof out[n].name, "%s", g->prof[i].name);
        out[n].ms = ms;
        n++;
    }
    return n;
}

ttc_status ttc_load_ex(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                       const ttc_load_opts *opts, ttc_graph **out) {
    if (!out) {
        set_last_error("out is NULL");
        return TTC_ERR_INVALID;
    }
    *out = nullptr;
    if (m && (!src || !dst || !t)) {
        set_last_error("src, dst and t must be non-NULL when m > 0");
        return TTC_ERR_INVALID;
    }
    ttc_graph *g = nullptr;
    TTC_API_BEGIN
    LoadOptions lo;
    if (opts) {
        lo.flags = opts->flags;
        lo.orientation = opts->orientation;
        lo.labeling = opts->labeling;
        lo.light_max_pairs = opts->light_max_pairs;
        lo.heavy_warp_cap = opts->heavy_warp_cap;
        lo.heavy_cta_cap = opts->heavy_cta_cap;
        lo.heavy_merge = opts->heavy_merge;
        lo.seed = opts->seed;
        if (lo.heavy_merge > TTC_HEAVY_MERGE) fail(TTC_ERR_INVALID, "unknown heavy_merge %u", lo.heavy_merge);
        if (lo.flags & ~(TTC_LOAD_DEVICE_INPUT | TTC_LOAD_PROFILE | TTC_LOAD_STREAM | TTC_LOAD_STRICT_TIME))
            fail(TTC_ERR_INVALID, "unknown load flags 0x%x", lo.flags);
    }
    g = new ttc_graph();
    TTC_CUDA(cudaGetDevice(&g->device));
    if (opts && opts->stream) {
        g->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        TTC_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
        g->own_stream = true;
    }
    g->profiling = (lo.flags & TTC_LOAD_PROFILE) != 0;
    build_graph(g, src, dst, t, m, lo);
    g->st.device_bytes = graph_device_bytes(g);
    *out = g;
    return TTC_OK;
    }
    catch (const Failure &f) {
        set_last_error(f.message);
        graph_destroy(g);
        return f.status;
    }
    catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        graph_destroy(g);
        return TTC_ERR_NOMEM;
    }
    catch (...) {
        set_last_error("unexpected internal failure");
        graph_destroy(g);
        return TTC_ERR_INTERNAL;
    }
}

ttc_graph *ttc_load(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m) {
    ttc_graph *g = nullptr;
    return ttc_load_ex(src, dst, t, m, nullptr, &g) == TTC_OK ? g : nullptr;
}

void ttc_free(ttc_graph *g) { graph_destroy(g); }

ttc_status ttc_graph_info(const ttc_graph *g, ttc_graph_stats *s) {
    if (!g || !s) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    *s = g->st;
    s->device_bytes = graph_device_bytes(g);
    return TTC_OK;
}

ttc_status ttc_count(ttc_graph *g, const ttc_delta *d, uint64_t out[TTC_NUM_TYPES]) {
    if (!g || !d || !out) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    TTC_API_BEGIN
    return run_queries(g, d, 1, out);
    TTC_API_END
}

ttc_status ttc_count_batch(ttc_graph *g, const ttc_delta *d, uint32_t k, uint64_t *out) {
    if (!g || (k && (!d || !out))) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (!k) return TTC_OK;
    TTC_API_BEGIN
    return run_queries(g, d, k, out);
    TTC_API_END
}

ttc_status ttc_count_shard(ttc_graph *g, const ttc_delta *d, uint32_t k, uint32_t shard, uint32_t nshards,
                           uint64_t *out) {
    if (!g || (k && (!d || !out))) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (!nshards || shard >= nshards) {
        set_last_error("shard " + std::to_string(shard) + " of " + std::to_string(nshards) + " does not exist");
        return TTC_ERR_INVALID;
    }
    if (g->streamed) {
        set_last_error("the graph was loaded with TTC_LOAD_STREAM: it keeps no triangle list to divide");
        return TTC_ERR_INVALID;
    }
    if (!k) return TTC_OK;
    TTC_API_BEGIN
    return run_queries(g, d, k, out, shard, nshards);
    TTC_API_END
}

ttc_status ttc_count_grid(ttc_graph *g, int64_t d13, const int64_t *d12, uint32_t n12, const int64_t *d23,
                          uint32_t n23, uint64_t *out, double *cyclic) {
    if (!g || (n12 && n23 && (!d12 || !d23 || !out))) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    const uint64_t k = (uint64_t)n12 * n23;
    if (!k) return TTC_OK;
    if (k > (uint64_t(1) << 20)) {
        set_last_error("grid of " + std::to_string(k) + " points exceeds 2^20");
        return TTC_ERR_RANGE;
    }
    TTC_API_BEGIN
    std::vector<ttc_delta> d(k);
    for (uint32_t i = 0; i < n12; i++)
        for (uint32_t j = 0; j < n23; j++) d[(size_t)i * n23 + j] = ttc_delta{d13, d12[i], d23[j]};
    const ttc_status rc = run_queries(g, d.data(), (uint32_t)k, out);
    if (rc == TTC_OK && cyclic) {
        for (uint64_t q = 0; q < k; q++) {
            const uint64_t *c = out + 8 * q;
            long double tot = 0;
            for (int t = 0; t < 8; t++) tot += (long double)c[t];
            cyclic[q] = tot > 0 ? (double)(((long double)c[3] + (long double)c[7]) / tot) : 0.0;
        }
    }
    return rc;
    TTC_API_END
}

ttc_status ttc_count_batch_async(ttc_graph *g, const ttc_delta *d_dev, uint32_t k, uint64_t *out_dev,
                                 void *stream) {
    if (!g || (k && (!d_dev || !out_dev))) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (!k) return TTC_OK;
    TTC_API_BEGIN
    TTC_CUDA(cudaSetDevice(g->device));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g->stream;
    TTC_CUDA(cudaMemsetAsync(out_dev, 0, 8 * (size_t)k * 8, s));
    DevBuf<int64_t> dq(3 * (size_t)k, s);  // freed in stream order after the kernels
    TTC_CUDA(cudaMemcpyAsync(dq.get(), d_dev, 3 * (size_t)k * 8, cudaMemcpyDeviceToDevice, s));
    normalise_kernel<<<(k + 127) / 128, 128, 0, s>>>(dq.get(), k);
    TTC_LAUNCH_CHECK();
    std::lock_guard<std::mutex> lock(g->mu);
    prof_reset(g);
    count_queue(g, dq.get(), k, reinterpret_cast<unsigned long long *>(out_dev), s);
    return TTC_OK;
    TTC_API_END
}

ttc_status ttc_count_multi(ttc_graph *const *g, const ttc_delta *d, uint32_t G, uint64_t *out) {
    if (G && (!g || !d || !out)) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    TTC_API_BEGIN
    // graphs loaded with TTC_LOAD_STREAM keep no triangle list to share:
    // the listed ones run in the shared launch, the streamed ones one by one
    std::vector<ttc_graph *> listed;
    std::vector<ttc_delta> ld;
    std::vector<uint32_t> where, streamed;
    for (uint32_t i = 0; i < G; i++) {
        if (g[i] && g[i]->streamed) {
            streamed.push_back(i);
        } else {
            listed.push_back(g[i]);
            ld.push_back(d[i]);
            where.push_back(i);
        }
    }
    if (streamed.empty()) {
        count_multi(g, d, G, out);
        return TTC_OK;
    }
    if (!listed.empty()) {
        std::vector<uint64_t> lo(8 * listed.size());
        count_multi(listed.data(), ld.data(), (uint32_t)listed.size(), lo.data());
        for (size_t j = 0; j < where.size(); j++) memcpy(out + 8 * (size_t)where[j], &lo[8 * j], 64);
    }
    for (uint32_t i : streamed) {
        const ttc_status rc = run_queries(g[i], d + i, 1, out + 8 * (size_t)i);
        if (rc != TTC_OK) return rc;
    }
    return TTC_OK;
    TTC_API_END
}

ttc_status ttc_count_sample(ttc_graph *g, const ttc_delta *d, uint64_t first, uint64_t stride, uint64_t cap,
                            uint32_t *tri, uint64_t *out, uint64_t *written) {
    if (!g || !d || !written || (cap && (!tri || !out)) || !stride) {
        set_last_error("NULL argument or zero stride");
        return TTC_ERR_INVALID;
    }
    if (g->streamed) {
        set_last_error("the graph was loaded with TTC_LOAD_STREAM: it keeps no triangle list to sample");
        return TTC_ERR_INVALID;
    }
    TTC_API_BEGIN
    int64_t hq[3];
    normalise(*d, hq);
    std::lock_guard<std::mutex> lock(g->mu);
    TTC_CUDA(cudaSetDevice(g->device));
    DevBuf<int64_t> dq(3, g->stream);
    TTC_CUDA(cudaMemcpyAsync(dq.get(), hq, 24, cudaMemcpyHostToDevice, g->stream));
    count_sample(g, dq.get(), first, stride, cap, tri, reinterpret_cast<unsigned long long *>(out), written);
    return TTC_OK;
    TTC_API_END
}

ttc_status ttc_count_participation(ttc_graph *g, const ttc_delta *d, uint64_t *vertex, uint64_t *pair) {
    if (!g || !d) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (g->streamed) {
        set_last_error("the graph was loaded with TTC_LOAD_STREAM: it keeps no triangle list");
        return TTC_ERR_INVALID;
    }
    TTC_API_BEGIN
    int64_t hq[3];
    normalise(*d, hq);
    std::lock_guard<std::mutex> lock(g->mu);
    TTC_CUDA(cudaSetDevice(g->device));
    DevBuf<int64_t> dq(3, g->stream);
    TTC_CUDA(cudaMemcpyAsync(dq.get(), hq, 24, cudaMemcpyHostToDevice, g->stream));
    count_participation(g, dq.get(), vertex, pair);
    return TTC_OK;
    TTC_API_END
}

ttc_status ttc_graph_pairs(ttc_graph *g, uint32_t *lohi) {
    if (!g || (g->st.m_s && !lohi)) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    TTC_API_BEGIN
    std::lock_guard<std::mutex> lock(g->mu);
    TTC_CUDA(cudaSetDevice(g->device));
    if (g->st.m_s) {
        TTC_CUDA(cudaMemcpyAsync(lohi, g->pair_vtx.get(), g->st.m_s * 8, cudaMemcpyDeviceToHost, g->stream));
        TTC_CUDA(cudaStreamSynchronize(g->stream));
    }
    return TTC_OK;
    TTC_API_END
}

}  // extern "C"
