// ttc_count_multi: many resident graphs counted in one launch.
//
// A plan is built once per ordered set of graph handles: a device table of
// the graphs (GraphView), exclusive prefixes over the graphs of their light
// chunks and heavy records, per-graph delta and count slots, and scratch for
// any graph with huge triangles.  The light kernel and the one-CTA-per-
// triangle heavy kernel then each run once over all graphs (persistent grids
// sized to the GPU), followed by the flat path of any graph with huge
// triangles.  The whole sequence, including the delta upload and the count
// download, is captured into a CUDA graph and replayed on later calls.
//
// The grid shapes (light CTAs per SM, heavy CTAs per SM) are chosen by a
// small autotuner: on first use of a plan every candidate is timed on the
// real graphs and the fastest is kept; results are cached per (GPU, plan
// shape) in a JSON file ($TTC_TUNE_CACHE, default ~/.cache/ttc/tune.json).
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "graph.cuh"

namespace ttc {
void set_last_error(const std::string &m);
void normalise(const ttc_delta &d, int64_t out[3]);

}  // namespace ttc

using namespace ttc;

namespace {

struct Shape {
    int light_per_sm = 8, heavy_per_sm = 2;
    int extra = 0;  // heavy-caps entries: the one-CTA class's search form (0 = none recorded)
};

// ---------------------------------------------------------------- tune cache
std::mutex g_tune_mu;

std::string tune_path() {
    const char *p = getenv("TTC_TUNE_CACHE");
    if (p && *p) return p;
    const char *home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/ttc/tune.json";
}

// The cache is a flat JSON object {"key": [light, heavy], ...}; an entry may
// carry a third number (Shape::extra).
std::map<std::string, Shape> tune_load() {
    std::map<std::string, Shape> m;
    std::ifstream f(tune_path());
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while ((i = s.find('"', i)) != std::string::npos) {
        const size_t j = s.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = s.substr(i + 1, j - i - 1);
        const size_t a = s.find('[', j), b = s.find(']', j);
        if (a == std::string::npos || b == std::string::npos) break;
        Shape sh;
        const int got = sscanf(s.c_str() + a + 1, "%d , %d , %d", &sh.light_per_sm, &sh.heavy_per_sm, &sh.extra);
        if (got < 3) sh.extra = 0;
        if (got >= 2 && sh.light_per_sm > 0 && (sh.heavy_per_sm > 0 || key.rfind("light|", 0) == 0))
            m[key] = sh;
        i = b + 1;
    }
    return m;
}

void tune_store(const std::map<std::string, Shape> &m) {
    const std::string path = tune_path();
    std::string dir = path.substr(0, path.rfind('/'));
    for (size_t k = 1; k <= dir.size(); k++)
        if (k == dir.size() || dir[k] == '/') mkdir(dir.substr(0, k).c_str(), 0755);
    const std::string tmp = path + ".tmp";
    std::ofstream f(tmp);
    if (!f) return;
    f << "{";
    bool first = true;
    for (auto &kv : m) {
        f << (first ? "\n" : ",\n") << "  \"" << kv.first << "\": [" << kv.second.light_per_sm << ", "
          << kv.second.heavy_per_sm;
        if (kv.second.extra) f << ", " << kv.second.extra;
        f << "]";
        first = false;
    }
    f << "\n}\n";
    f.close();
    rename(tmp.c_str(), path.c_str());
}

// ---------------------------------------------------------------- light threshold
// Graphs are tuned by shape: the GPU's SM count and the bit lengths of m,
// m_s, the largest multiplicity and kappa.  The cache keeps
// "light|..." keys as [threshold, 0].
std::map<std::string, Shape> g_light_mem;  // guarded by g_tune_mu; loaded once
bool g_light_loaded = false;

std::string light_key(const ttc_graph_stats &st) {
    char b[128];
    snprintf(b, sizeof b, "light|sm%d|m%d|s%d|x%d|k%d", sm_count(), bits_for(st.m), bits_for(st.m_s),
             bits_for(st.sigma_max), bits_for(st.kappa));
    return b;
}

// The heavy-class caps are tuned for a shape and the light threshold in use
// (which decides the heavy triangles): "heavy|...|l<threshold>" keys as
// [warp cap, CTA cap].
std::string heavy_key(const ttc_graph_stats &st, uint32_t light) {
    char b[160];
    snprintf(b, sizeof b, "heavy|sm%d|m%d|s%d|x%d|k%d|l%u", sm_count(), bits_for(st.m), bits_for(st.m_s),
             bits_for(st.sigma_max), bits_for(st.kappa), light);
    return std::string(b);
}

// ---------------------------------------------------------------- plans
struct Plan {
    std::vector<ttc_graph *> graphs;
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t G = 0;
    MultiTable table{};
    DevBuf<GraphView> gv;
    DevBuf<uint64_t> chunk_pre, hwarp_pre, hcta_pre;
    DevBuf<int64_t> dq;
    DevBuf<unsigned long long> acc;  // [G][8] + overflow flag
    std::vector<DevBuf<uint8_t>> huge_scratch;
    int64_t *h_dq = nullptr;             // pinned
    unsigned long long *h_acc = nullptr;  // pinned
    Shape shape;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;

    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (stream) cudaStreamSynchronize(stream);
        gv.reset(); chunk_pre.reset(); hwarp_pre.reset(); hcta_pre.reset(); dq.reset(); acc.reset();
        huge_scratch.clear();
        if (h_dq) cudaFreeHost(h_dq);
        if (h_acc) cudaFreeHost(h_acc);
        if (stream) cudaStreamDestroy(stream);
    }

    // everything one count needs, queued on `stream`
    void enqueue(const Shape &sh) {
        cudaStream_t s = stream;
        TTC_CUDA(cudaMemcpyAsync(dq.get(), h_dq, 3 * (size_t)G * 8, cudaMemcpyHostToDevice, s));
        TTC_CUDA(cudaMemsetAsync(acc.get(), 0, (8 * (size_t)G + 1) * 8, s));
        count_multi_launch(table, dq.get(), acc.get(), sh.light_per_sm, sh.heavy_per_sm, s);
        for (uint32_t i = 0, k = 0; i < G; i++) {
            ttc_graph *g = graphs[i];
            if (!g->st.tau_huge) continue;
            count_huge_of(g, dq.get() + 3 * (size_t)i, acc.get() + 8 * (size_t)i, acc.get() + 8 * (size_t)G,
                          huge_scratch[k++].get(), s);
        }
        TTC_CUDA(cudaMemcpyAsync(h_acc, acc.get(), (8 * (size_t)G + 1) * 8, cudaMemcpyDeviceToHost, s));
    }

    std::string tune_key() const {
        int sms = sm_count();
        cudaDeviceProp prop{};
        cudaGetDeviceProperties(&prop, device);
        char buf[512];
        snprintf(buf, sizeof buf, "%s|sm%d|G%d|c%d|h%d|w%d", prop.name, sms, (int)std::log2((double)G + 1),
                 (int)std::log2((double)table.chunks + 1), (int)std::log2((double)(table.hwarp + table.hcta) + 1),
                 table.any_wide);
        std::string k = buf;
        std::replace(k.begin(), k.end(), '"', '\'');
        return k;
    }

    // time every candidate shape on the real graphs and keep the fastest
    void autotune() {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto cache = tune_load();
        const std::string key = tune_key();
        auto it = cache.find(key);
        if (it != cache.end()) {
            shape = it->second;
            return;
        }
        cudaEvent_t a, b;
        TTC_CUDA(cudaEventCreate(&a));
        TTC_CUDA(cudaEventCreate(&b));
        float best = 1e30f;
        for (int lp : {4, 8, 16}) {
            for (int hp : {1, 2, 4}) {
                if (!(table.hwarp + table.hcta) && hp != 2) continue;
                const Shape sh{lp, hp};
                enqueue(sh);  // warm
                TTC_CUDA(cudaEventRecord(a, stream));
                for (int r = 0; r < 2; r++) enqueue(sh);
                TTC_CUDA(cudaEventRecord(b, stream));
                TTC_CUDA(cudaEventSynchronize(b));
                float ms = 0;
                TTC_CUDA(cudaEventElapsedTime(&ms, a, b));
                if (ms < best) {
                    best = ms;
                    shape = sh;
                }
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cache[key] = shape;
        tune_store(cache);
    }

    void capture() {
        cudaGraph_t graph;
        TTC_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue(shape);
        } catch (...) {
            cudaStreamEndCapture(stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        TTC_CUDA(cudaStreamEndCapture(stream, &graph));
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TTC_CUDA(e);
    }
};

std::mutex g_plan_mu;
std::vector<std::unique_ptr<Plan>> g_plans;
uint64_t g_plan_clock = 0;
constexpr size_t MAX_PLANS = 4;

Plan *build_plan(ttc_graph *const *gs, uint32_t G) {
    auto p = std::make_unique<Plan>();
    p->graphs.assign(gs, gs + G);
    p->G = G;
    TTC_CUDA(cudaGetDevice(&p->device));
    TTC_CUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
    cudaStream_t s = p->stream;
    std::vector<GraphView> views(G);
    std::vector<uint64_t> cpre(G + 1, 0), wpre(G + 1, 0), hpre(G + 1, 0);
    MultiTable &t = p->table;
    for (uint32_t i = 0; i < G; i++) {
        ttc_graph *g = gs[i];
        if (g->device != p->device) fail(TTC_ERR_INVALID, "graph %u lives on another device", i);
        if (g->strict != gs[0]->strict)
            fail(TTC_ERR_INVALID, "graph %u reads ties differently (TTC_LOAD_STRICT_TIME) from graph 0", i);
        t.strict = gs[0]->strict;
        // make sure the graph's own stream has finished building it
        TTC_CUDA(cudaStreamSynchronize(g->stream));
        views[i] = g->view_host;
        cpre[i + 1] = cpre[i] + (g->st.tau_light + 31) / 32;
        wpre[i + 1] = wpre[i] + g->st.tau_hwarp;
        hpre[i + 1] = hpre[i] + g->st.tau_hcta;
        if (g->st.tau_hwarp + g->st.tau_hcta) (g->heavy_wide ? t.any_wide : t.any_narrow) = 1;
        if (g->st.tau_huge) {
            p->huge_scratch.emplace_back();
            p->huge_scratch.back().alloc(heavy_scratch_bytes(g), s);
        }
    }
    p->gv.alloc(G, s);
    p->chunk_pre.alloc(G + 1, s);
    p->hwarp_pre.alloc(G + 1, s);
    p->hcta_pre.alloc(G + 1, s);
    p->dq.alloc(3 * (size_t)G, s);
    p->acc.alloc(8 * (size_t)G + 1, s);
    TTC_CUDA(cudaMemcpyAsync(p->gv.get(), views.data(), sizeof(GraphView) * G, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemcpyAsync(p->chunk_pre.get(), cpre.data(), 8 * (G + 1), cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemcpyAsync(p->hwarp_pre.get(), wpre.data(), 8 * (G + 1), cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemcpyAsync(p->hcta_pre.get(), hpre.data(), 8 * (G + 1), cudaMemcpyHostToDevice, s));
    t.gvs = p->gv.get();
    t.G = G;
    t.chunk_pre = p->chunk_pre.get();
    t.hwarp_pre = p->hwarp_pre.get();
    t.hcta_pre = p->hcta_pre.get();
    t.chunks = cpre[G];
    t.hwarp = wpre[G];
    t.hcta = hpre[G];
    TTC_CUDA(cudaMallocHost(&p->h_dq, 3 * (size_t)G * 8));
    TTC_CUDA(cudaMallocHost(&p->h_acc, (8 * (size_t)G + 1) * 8));
    TTC_CUDA(cudaStreamSynchronize(s));
    return p.release();
}

}  // namespace

namespace ttc {

// Drops every cached plan that names g (called before g is freed).
void multi_forget(ttc_graph *g) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plans.erase(std::remove_if(g_plans.begin(), g_plans.end(),
                                 [&](const std::unique_ptr<Plan> &p) {
                                     return std::find(p->graphs.begin(), p->graphs.end(), g) != p->graphs.end();
                                 }),
                  g_plans.end());
}

void count_multi(ttc_graph *const *gs, const ttc_delta *d, uint32_t G, uint64_t *out) {
    if (!G) return;
    std::vector<int64_t> hq(3 * (size_t)G);
    for (uint32_t i = 0; i < G; i++) {
        if (!gs[i]) fail(TTC_ERR_INVALID, "graph %u is NULL", i);
        normalise(d[i], &hq[3 * (size_t)i]);
    }
    std::lock_guard<std::mutex> lock(g_plan_mu);
    Plan *plan = nullptr;
    for (auto &p : g_plans)
        if (p->G == G && std::equal(p->graphs.begin(), p->graphs.end(), gs)) plan = p.get();
    if (!plan) {
        if (g_plans.size() >= MAX_PLANS) {
            auto oldest = std::min_element(g_plans.begin(), g_plans.end(),
                                           [](const std::unique_ptr<Plan> &a, const std::unique_ptr<Plan> &b) {
                                               return a->last_use < b->last_use;
                                           });
            g_plans.erase(oldest);
        }
        std::unique_ptr<Plan> p(build_plan(gs, G));
        memcpy(p->h_dq, hq.data(), hq.size() * 8);
        p->autotune();
        p->capture();
        g_plans.push_back(std::move(p));
        plan = g_plans.back().get();
    }
    plan->last_use = ++g_plan_clock;
    TTC_CUDA(cudaSetDevice(plan->device));
    memcpy(plan->h_dq, hq.data(), hq.size() * 8);
    TTC_CUDA(cudaGraphLaunch(plan->exec, plan->stream));
    note_launch();
    TTC_CUDA(cudaStreamSynchronize(plan->stream));
    check_count_flag(plan->h_acc[8 * (size_t)G]);
    memcpy(out, plan->h_acc, 8 * (size_t)G * 8);
}

}  // namespace ttc

namespace ttc {

uint32_t tuned_light_max(const ttc_graph_stats &st) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_light_loaded) {
        g_light_mem = tune_load();
        g_light_loaded = true;
    }
    const auto it = g_light_mem.find(light_key(st));
    return it != g_light_mem.end() ? (uint32_t)it->second.light_per_sm : default_light_max_pairs();
}

bool tuned_heavy_caps(const ttc_graph_stats &st, uint32_t light, uint32_t *warp_cap, uint32_t *cta_cap,
                      uint32_t *merge) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_light_loaded) {
        g_light_mem = tune_load();
        g_light_loaded = true;
    }
    const auto it = g_light_mem.find(heavy_key(st, light));
    if (it == g_light_mem.end()) return false;
    *warp_cap = (uint32_t)it->second.light_per_sm;
    *cta_cap = (uint32_t)it->second.heavy_per_sm;
    const int x = it->second.extra;
    *merge = x == (int)TTC_HEAVY_BINARY || x == (int)TTC_HEAVY_MERGE ? (uint32_t)x : 0u;
    return true;
}

namespace {

// Load plus one batched count of the probe queries, timed with CUDA events
// on the options' stream: one untimed run (first-use work), then the
// fastest of `timed` runs; st gets the graph's statistics.
ttc_status time_load_count(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                           const ttc_load_opts &o, const ttc_delta *probe, uint32_t k, int timed, float *best,
                           ttc_graph_stats *st) {
    std::vector<uint64_t> out(8 * (size_t)(k ? k : 1));
    for (int rep = 0; rep <= timed; rep++) {
        float ms = 0.f;
        float *el = &ms;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TTC_CUDA(cudaEventCreate(&e0));
        TTC_CUDA(cudaEventCreate(&e1));
        cudaStream_t s = static_cast<cudaStream_t>(o.stream);
        TTC_CUDA(cudaEventRecord(e0, s));
        ttc_graph *g = nullptr;
        ttc_status rc = ttc_load_ex(src, dst, t, m, &o, &g);
        if (rc == TTC_OK && k) rc = ttc_count_batch(g, probe, k, out.data());
        if (rc == TTC_OK) {
            *st = g->st;
            TTC_CUDA(cudaStreamSynchronize(g->stream));
        }
        ttc_free(g);
        TTC_CUDA(cudaEventRecord(e1, s));
        TTC_CUDA(cudaEventSynchronize(e1));
        TTC_CUDA(cudaEventElapsedTime(el, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != TTC_OK) return rc;
        if (rep == 1 || (rep > 1 && ms < *best)) *best = ms;
    }
    return TTC_OK;
}

}  // namespace

}  // namespace ttc

extern "C" ttc_status ttc_tune_light(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                                     const ttc_load_opts *opts, const ttc_delta *probe, uint32_t k,
                                     uint32_t *chosen, float *ms) {
    if (!chosen || (k && !probe)) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (opts && opts->light_max_pairs) {
        set_last_error("ttc_tune_light chooses light_max_pairs itself: pass 0");
        return TTC_ERR_INVALID;
    }
    try {
        ttc_load_opts o = opts ? *opts : ttc_load_opts{};
        float best = 0.f;
        uint32_t best_c = default_light_max_pairs();
        ttc_graph_stats st{};
        for (uint32_t i = 0; i < TTC_TUNE_CANDIDATES; i++) {
            o.light_max_pairs = ttc_tune_candidates[i];
            float el = 0.f;
            const ttc_status rc = time_load_count(src, dst, t, m, o, probe, k, 2, &el, &st);
            if (rc != TTC_OK) return rc;
            if (ms) ms[i] = el;
            if (i == 0 || el < best) {
                best = el;
                best_c = ttc_tune_candidates[i];
            }
        }
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto cache = tune_load();
            Shape sh;
            sh.light_per_sm = (int)best_c;
            sh.heavy_per_sm = 0;
            cache[light_key(st)] = sh;
            tune_store(cache);
            g_light_mem = cache;
            g_light_loaded = true;
        }
        *chosen = best_c;
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    } catch (...) {
        set_last_error("unexpected internal failure");
        return TTC_ERR_INTERNAL;
    }
}

extern "C" ttc_status ttc_tune_heavy(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                                     const ttc_load_opts *opts, const ttc_delta *probe, uint32_t k,
                                     uint32_t *warp_cap, uint32_t *cta_cap, uint32_t *merge, float *ms) {
    if (!warp_cap || !cta_cap || !merge || (k && !probe)) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (opts && (opts->heavy_warp_cap || opts->heavy_cta_cap || opts->heavy_merge)) {
        set_last_error("ttc_tune_heavy chooses the heavy caps and search form itself: pass 0");
        return TTC_ERR_INVALID;
    }
    try {
        ttc_load_opts o = opts ? *opts : ttc_load_opts{};
        float best = 0.f;
        uint32_t bw = 0, bc = 0, bm = 0, dw = 0, dc = 0, dm = 0;
        ttc_graph_stats st{};
        for (uint32_t i = 0; i < TTC_TUNE_HEAVY_CANDIDATES; i++) {
            o.heavy_warp_cap = ttc_tune_heavy_candidates[i][0];
            o.heavy_cta_cap = ttc_tune_heavy_candidates[i][1];
            o.heavy_merge = ttc_tune_heavy_candidates[i][2];
            float el = 0.f;
            const ttc_status rc = time_load_count(src, dst, t, m, o, probe, k, 3, &el, &st);
            if (rc != TTC_OK) return rc;
            if (ms) ms[i] = el;
            // another candidate replaces the first (the kernels' capacities,
            // binary searches) only when it is faster by more than 1%, not by
            // timing noise
            if (i == 0) {
                dw = st.heavy_warp_cap;
                dc = st.heavy_cta_cap;
                dm = st.heavy_merge;
            }
            if (i == 0 || el < best * (bw == dw && bc == dc && bm == dm ? 0.99f : 1.0f)) {
                best = el;
                bw = st.heavy_warp_cap;
                bc = st.heavy_cta_cap;
                bm = st.heavy_merge;
            }
            if (!st.tau_heavy) {  // no heavy triangle: every candidate counts the same
                for (uint32_t j = i + 1; ms && j < TTC_TUNE_HEAVY_CANDIDATES; j++) ms[j] = el;
                break;
            }
        }
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto cache = tune_load();
            Shape sh;
            sh.light_per_sm = (int)bw;
            sh.heavy_per_sm = (int)bc;
            sh.extra = (int)bm;
            cache[heavy_key(st, st.light_max_pairs)] = sh;
            tune_store(cache);
            g_light_mem = cache;
            g_light_loaded = true;
        }
        *warp_cap = bw;
        *cta_cap = bc;
        *merge = bm;
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    } catch (...) {
        set_last_error("unexpected internal failure");
        return TTC_ERR_INTERNAL;
    }
}

extern "C" ttc_status ttc_count_stream(const uint32_t *const *src, const uint32_t *const *dst,
                                       const int64_t *const *t, const uint64_t *m, const ttc_delta *d, uint32_t G,
                                       const ttc_load_opts *opts, uint64_t budget_bytes, uint64_t *out,
                                       uint32_t *batches) {
    if (G && (!src || !dst || !t || !m || !d || !out)) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (opts && (opts->flags & (TTC_LOAD_DEVICE_INPUT | TTC_LOAD_STREAM))) {
        set_last_error("ttc_count_stream loads host arrays into listed graphs: "
                       "TTC_LOAD_DEVICE_INPUT and TTC_LOAD_STREAM are refused");
        return TTC_ERR_INVALID;
    }
    std::vector<ttc_graph *> batch;
    uint32_t first = 0, nb = 0;  // first graph of the current batch
    auto release = [&]() {
        for (ttc_graph *g : batch) ttc_free(g);
        batch.clear();
    };
    auto flush = [&]() -> ttc_status {
        if (batch.empty()) return TTC_OK;
        const ttc_status rc = ttc_count_multi(batch.data(), d + first, (uint32_t)batch.size(), out + 8 * (size_t)first);
        release();
        nb++;
        return rc;
    };
    uint64_t budget = budget_bytes, bytes = 0;
    if (!budget) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("cudaMemGetInfo failed");
            return TTC_ERR_CUDA;
        }
        budget = fr / 2;
    }
    for (uint32_t i = 0; i < G; i++) {
        ttc_graph *g = nullptr;
        ttc_status rc = ttc_load_ex(src[i], dst[i], t[i], m[i], opts, &g);
        if (rc == TTC_ERR_NOMEM && !batch.empty()) {
            // the resident batch may be what left too little room: count and
            // free it, then load the graph again into the memory it held
            rc = flush();
            if (rc != TTC_OK) return rc;
            first = i;
            bytes = 0;
            rc = ttc_load_ex(src[i], dst[i], t[i], m[i], opts, &g);
        }
        if (rc != TTC_OK) {
            release();
            return rc;
        }
        const uint64_t b = g->st.device_bytes;
        if (!batch.empty() && bytes + b > budget) {
            rc = flush();
            if (rc != TTC_OK) {
                ttc_free(g);
                return rc;
            }
            first = i;
            bytes = 0;
        }
        batch.push_back(g);
        bytes += b;
    }
    const ttc_status rc = flush();
    if (batches) *batches = nb;
    return rc;
}
