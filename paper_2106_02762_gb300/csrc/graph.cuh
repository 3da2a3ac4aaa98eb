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

struct ttc_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ttc_graph_stats st{};
    uint32_t labeling = 0;
    uint32_t light_max_pairs = 0;

    int64_t tmin = 0;   // smallest timestamp
    int64_t span = 0;   // largest minus smallest timestamp
    int shift = 1;      // see key layout above

    ttc::DevBuf<int64_t> key;     // [m]
    ttc::DevBuf<uint32_t> fwd;    // [m + 1] exclusive prefix of (stored dir == 0)
    ttc::DevBuf<uint32_t> poff;   // [m_s + 1] first edge of each pair
    ttc::DevBuf<uint2> pair_vtx;  // [m_s] (smaller id, larger id) of each pair
    ttc::DevBuf<uint4> tri;       // [tau] light records first, then heavy ones
    // prefix-sum (CEC) path for heavy triangles
    ttc::DevBuf<uint64_t> heavy_eoff;  // [tau_heavy + 1] enumerated-element offsets
    int heavy_wide = 0;                // 1: 64-bit prefix sums needed
    uint64_t heavy_elems = 0;

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

// count.cu: the same kernels as count_queue for one normalised query, but
// with every device buffer supplied by the caller: acc (9 u64, zeroed by the
// caller) and the heavy-path prefix scratch of heavy_scratch_bytes(g) bytes.
// Allocates nothing.
size_t heavy_scratch_bytes(const ttc_graph *g);
void count_one_into(ttc_graph *g, const int64_t *dq, unsigned long long *acc, void *scratch, cudaStream_t s);

// count.cu: per-triangle counts of a strided sample of the triangle list.
// (host outputs; the sampled triangles run through the same light/heavy code)
void count_sample(ttc_graph *g, const int64_t *dq, uint64_t first, uint64_t stride, uint64_t cap,
                  uint32_t *tri_vtx_host, unsigned long long *out_host, uint64_t *written);

// count.cu: many graphs in one persistent launch.
struct MultiGraphDesc;
void count_multi_launch(const MultiGraphDesc *descs_dev, uint32_t G, const uint64_t *tri_prefix_dev,
                        uint64_t tri_total, unsigned long long *acc, cudaStream_t s);

uint32_t default_light_max_pairs();

}  // namespace ttc
