// The device-resident graph built by ttc_load and read by the count kernels.
#pragma once

#include <mutex>

#include "common.cuh"

// Per-edge packed key (one int64 per temporal edge, grouped by vertex pair):
//   key = (t - t_min) << shift | tie_rank << 1 | dir
// where tie_rank is the edge's rank among edges with the same timestamp
// (ordered by input index), so key order is the (t, index) order of the
// paper's edges, and dir = 1 when the edge runs from the pair's larger vertex
// id to its smaller one.  Keys fit in 63 bits (checked at load).
//
// Triangle record (uint4): x = pair A, y = pair B, z = pair C, w = flags.
// The triangle's vertices are named u, v, w so that A = {u, v}, B = {u, w},
// C = {v, w}; C is the pair that is only searched, A and B are enumerated
// (Sec. 5).  In the kernels "direction 0" means u->v on A, u->w on B and
// v->w on C; flag bit i (i = 0, 1, 2 for A, B, C) says the stored dir bit is
// the opposite of that.
struct TriRec {
    static constexpr uint32_t FLIP_A = 1u, FLIP_B = 2u, FLIP_C = 4u;
};

// What the count kernels see of one resident graph (plain pointers; an array
// of these is the "graph table" of a many-graph launch).
struct GraphView {
    const int64_t *key;
    const uint32_t *fwd;
    const uint32_t *poff;
    // records in bin order: light [0, n_light), then heavy ones for one warp
    // each (n_hwarp), for one CTA each (n_hcta), and the huge ones last;
    // n_heavy counts all three heavy bins
    const uint4 *tri;
    uint64_t n_light, n_hwarp, n_hcta, n_heavy;
    int64_t span;
    int shift;
    int wide;  // 64-bit prefix sums needed (some list has >= 65536 edges)
    int strict;  // TTC_LOAD_STRICT_TIME: a triple counts only if its times strictly increase
    uint64_t m, ms;  // lengths of key (edges) and of the pair arrays (for index checks)
};

struct ttc_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the count's heavy bins run on a second stream beside the light bin
    // (created at the first count; forked from and joined to the count's
    // stream by the two events)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    ttc_graph_stats st{};
    uint32_t labeling = 0;
    uint32_t light_max_pairs = 0;
    bool strict = false;  // TTC_LOAD_STRICT_TIME

    int64_t tmin = 0;   // smallest timestamp
    int64_t span = 0;   // largest minus smallest timestamp
    int shift = 1;      // see key layout above

    ttc::DevBuf<int64_t> key;     // [m]
    ttc::DevBuf<uint32_t> fwd;    // [m + 1] exclusive prefix of (stored dir == 0)
    ttc::DevBuf<uint32_t> poff;   // [m_s + 1] first edge of each pair
    ttc::DevBuf<uint2> pair_vtx;  // [m_s] (smaller id, larger id) of each pair
    ttc::DevBuf<uint4> tri;       // [tau] light records first, then heavy ones
    int heavy_wide = 0;           // 1: 64-bit prefix sums needed
    // heavy triangles too large for one CTA (flat prefix-sum path): the last
    // tau_huge records
    ttc::DevBuf<uint64_t> huge_eoff;    // [tau_huge + 1] enumerated-edge offsets
    uint64_t huge_elems = 0;
    // TTC_LOAD_STREAM: no light records; the oriented CSR and the
    // enumeration's work items are kept and each count enumerates again
    bool streamed = false;
    ttc::DevBuf<uint2> s_items;     // [s_nitems] (target v, first in-edge)
    uint32_t s_nitems = 0;
    ttc::DevBuf<uint4> s_ocsr;      // [m_s] per oriented edge: target rank, sigma word, pair
    ttc::DevBuf<uint32_t> s_onbr, s_osrc, s_in_e;  // [m_s]
    ttc::DevBuf<uint32_t> s_out_off, s_in_off;     // [n + 1]
    std::vector<uint32_t> s_chunks;  // work-item boundaries of the collecting passes
    uint64_t s_chunk_cap = 0;        // light records one collecting pass can hold
    // the graph as a one-entry graph table
    GraphView view_host{};
    ttc::DevBuf<GraphView> view;        // [1]
    ttc::DevBuf<uint64_t> prefix;       // [6]: {0, light chunks, 0, n_hwarp, 0, n_hcta}

    // sharded counts: per-bin views of one shard, and the huge offsets
    // (device copy of the shard's slice; host copy of the whole array)
    ttc::DevBuf<GraphView> shard_view;   // [3]
    ttc::DevBuf<uint64_t> shard_pre;     // [6]
    ttc::DevBuf<uint64_t> shard_eoff;    // [tau_huge + 1]
    std::vector<uint64_t> huge_eoff_host;

    // per-call device scratch, guarded by `mu`
    std::mutex mu;
    ttc::DevBuf<unsigned long long> acc;  // [cap * 8 + 1]: counts and the overflow flag
    ttc::DevBuf<int64_t> dq;              // [cap * 3] deltas
    ttc::DevBuf<uint8_t> scratch;         // heavy-path prefix arrays
    uint32_t acc_cap = 0;

    // optional per-kernel timing of count calls
    bool profiling = false;
    struct ProfEntry {
        const char *name;
        cudaEvent_t start, stop;
    };
    std::vector<ProfEntry> prof;  // events, reused across calls
    size_t prof_used = 0;
};

namespace ttc {

struct LoadOptions {
    uint32_t flags = 0, orientation = 0, labeling = 0, light_max_pairs = 0;
    uint32_t heavy_warp_cap = 0, heavy_cta_cap = 0, heavy_merge = 0;
    uint64_t seed = 0;
};

// load.cu: builds everything above (stream must already be set on g).
void build_graph(ttc_graph *g, const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                 const LoadOptions &opt);

// Profiling helpers: bracket one kernel launch with events when enabled.
void prof_reset(ttc_graph *g);
void prof_begin(ttc_graph *g, cudaStream_t s, const char *name);
void prof_end(ttc_graph *g, cudaStream_t s);

// count.cu: counts for k normalised delta-triples already on the device
// (dq: k * 3 int64 as d13, d12, d23), accumulated into acc ([k][8] u64 plus a
// trailing overflow flag), which the caller zeroes.
void count_queue(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s);
// The same for shard `shard` of `nshards`: the light, warp, CTA and huge
// records of the handle's bins are each cut into nshards consecutive slices
// of near-equal length, and only this shard's slices are counted.  Every
// static triangle lies in exactly one slice, so the shards' counts sum to
// count_queue's.  Not for TTC_LOAD_STREAM handles.
void count_queue_shard(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, uint32_t shard,
                       uint32_t nshards, cudaStream_t s);

// load.cu: for a TTC_LOAD_STREAM handle, the light triangles' counts for k
// normalised queries (dq on the device), added into acc ([k][8] plus the
// overflow flag): the enumeration runs again chunk by chunk of its work
// items, collects each chunk's light records into a buffer of
// s_chunk_cap records, and the light kernels count them for all k queries.
void stream_count_light(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s);
// Records per collecting buffer: TTC_STREAM_CHUNK from the environment, else
// 2^24 (at least the largest work item's room).
uint64_t stream_chunk_records();

// count.cu: the light kernels over the light records of the one-graph table
// view (pre: its 32-record chunk prefix {0, chunks}, both on the device);
// n_bound bounds the record count (sizes the grid).  k normalised queries,
// acc [k][8] plus the overflow flag.
void count_light_records(ttc_graph *g, const GraphView *view, const uint64_t *pre, uint64_t n_bound,
                         const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s);

// count.cu: the same kernels as count_queue for one normalised query, but
// with every device buffer supplied by the caller: acc (9 u64, zeroed by the
// caller) and the heavy-path prefix scratch of heavy_scratch_bytes(g) bytes.
// Allocates nothing.
size_t heavy_scratch_bytes(const ttc_graph *g);
// Queries one batched pass of the flat heavy path takes out of k (its
// scratch is that many times heavy_scratch_bytes(g)).
uint32_t huge_pass_queries(const ttc_graph *g, uint32_t k);
void count_one_into(ttc_graph *g, const int64_t *dq, unsigned long long *acc, void *scratch, cudaStream_t s);

// count.cu: per-triangle counts of a strided sample of the triangle list.
// (host outputs; the sampled triangles run through the same light/heavy code)
void count_participation(ttc_graph *g, const int64_t *dq, uint64_t *vertex_host, uint64_t *pair_host);
void count_sample(ttc_graph *g, const int64_t *dq, uint64_t first, uint64_t stride, uint64_t cap,
                  uint32_t *tri_vtx_host, unsigned long long *out_host, uint64_t *written);

// count.cu: many graphs in one launch of the light and heavy kernels over a
// device graph table; dq holds one normalised delta per graph; acc is [G][8]
// plus the overflow flag; light_per_sm / heavy_per_sm shape the grids.
struct MultiTable {
    const GraphView *gvs;
    uint32_t G;
    const uint64_t *chunk_pre, *hwarp_pre, *hcta_pre;  // exclusive prefixes over the graphs (G + 1)
    uint64_t chunks, hwarp, hcta;                       // their totals
    int any_narrow, any_wide;                           // prefix widths present in the heavy bins
    bool strict;                                        // TTC_LOAD_STRICT_TIME (all graphs alike)
};
void count_multi_launch(const MultiTable &t, const int64_t *dq, unsigned long long *acc, int light_per_sm,
                        int heavy_per_sm, cudaStream_t s);
// The flat path of one graph's huge triangles for one query (counts added to
// acc_row[8], overflow flag at *flag).
void count_huge_of(ttc_graph *g, const int64_t *dq_one, unsigned long long *acc_row, unsigned long long *flag,
                   void *scratch, cudaStream_t s);
// Largest A + B list length handled by one warp / one CTA of the heavy bin.
uint32_t warp_capacity(int wide);
uint32_t fused_capacity(int wide);

uint32_t default_light_max_pairs();
// multi.cu: the light threshold ttc_tune_light chose for graphs of this
// shape on the current GPU (the tune cache), else default_light_max_pairs().
uint32_t tuned_light_max(const ttc_graph_stats &st);
// The heavy-class caps tuned for graphs of this shape at light threshold
// `light` (ttc_tune_heavy), if any, and the one-CTA class's search form
// (TTC_HEAVY_*, 0 when the entry records none).
bool tuned_heavy_caps(const ttc_graph_stats &st, uint32_t light, uint32_t *warp_cap, uint32_t *cta_cap,
                      uint32_t *merge);

// A build with -DTTC_DEBUG_BOUNDS=1 checks the count kernels' indices on
// the device (count_dev.cuh); this returns and clears the device word those
// checks set (always 0 in other builds).
unsigned int take_bounds_word();

// Turns the count kernels' device flag word into a failure: bit 1 (a
// bounded wait in a kernel gave up) is TTC_ERR_TIMEOUT, any other bit (a
// carry out of a 64-bit count) TTC_ERR_OVERFLOW; 0 returns.
void check_count_flag(unsigned long long flag);

}  // namespace ttc
