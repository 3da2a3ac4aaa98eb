// ttc_load: everything of Alg. 1 that does not depend on the delta-triple.
//
//   a1 ingest      validate ids/timestamps, drop self-loops (Sec. 3)
//   a2 pairs       static graph G: group edges by vertex pair, multiplicity
//                  per pair, per-pair edge lists sorted by key (t, index)
//   a3 peel        degeneracy ordering by a bucketed parallel k-core peel
//                  (Sec. 3, Matula-Beck); one thread-block cluster runs every
//                  round, separated by cluster barriers
//   a4 orient      vertices renamed by rank in the ordering; DAG G< as an
//                  out-CSR (lists sorted by rank) and an in-CSR
//   a6 triangles   for each oriented edge u -> v: the part of N+(u) after v
//                  intersected with N+(v) (Sec. 5: u < v < w in the ordering)
//   records        per triangle the three pair ids, labelled for counting
//                  (which pair is only searched) and split into the light
//                  and heavy (prefix-sum) bins
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "graph.cuh"
#include "count_dev.cuh"
#include "sort.cuh"

namespace cg = cooperative_groups;

namespace ttc {

namespace {

constexpr int TPB = 256;
constexpr uint32_t UNSET = 0xffffffffu;

inline unsigned grid_for(size_t n, int tpb = TPB) {
    size_t b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    const size_t cap = (size_t)sm_count() * 32;
    return (unsigned)(b < cap ? b : cap);
}

#define GRID_STRIDE(i, n) \
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

struct IngestStats {
    unsigned long long loops;
    unsigned int max_id;
    unsigned int bad_id;
    unsigned int bad_t;
    unsigned int pad;
    long long tmin, tmax;  // over the kept edges
};

// Validates the input edges and flags self-loops.  src/dst/t may be device
// memory or page-locked host memory mapped into the device's address space;
// in the second case the kernel also writes the device copies (src_copy,
// dst_copy, t_copy non-null), so the input crosses the host link once.  Each
// thread loads INGEST_UNROLL elements before using any, so that many reads
// are in flight (host reads have a long latency).
constexpr int INGEST_UNROLL = 4;
__global__ void ingest_check_kernel(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                    const int64_t *__restrict__ t, size_t m, uint8_t *__restrict__ keep,
                                    IngestStats *st, uint32_t *__restrict__ src_copy, uint32_t *__restrict__ dst_copy,
                                    int64_t *__restrict__ t_copy) {
    const int64_t TLIM = (int64_t)1 << 62;
    unsigned int my_max = 0, bad_id = 0, bad_t = 0;
    unsigned long long loops = 0;
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += INGEST_UNROLL * stride) {
        uint32_t a[INGEST_UNROLL], b[INGEST_UNROLL];
        int64_t tt[INGEST_UNROLL];
#pragma unroll
        for (int k = 0; k < INGEST_UNROLL; k++) {
            const size_t i = i0 + k * stride;
            a[k] = i < m ? src[i] : 0u;
            b[k] = i < m ? dst[i] : 0u;
            tt[k] = i < m ? t[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < INGEST_UNROLL; k++) {
            const size_t i = i0 + k * stride;
            if (i >= m) break;
            if (src_copy) {
                src_copy[i] = a[k];
                dst_copy[i] = b[k];
                t_copy[i] = tt[k];
            }
            keep[i] = a[k] != b[k];
            loops += a[k] == b[k];
            if (a[k] != b[k]) {
                lo = min(lo, (long long)tt[k]);
                hi = max(hi, (long long)tt[k]);
            }
            my_max = max(my_max, max(a[k], b[k]));
            bad_id |= (a[k] >> 31) | (b[k] >> 31);
            bad_t |= (tt[k] < -TLIM) | (tt[k] > TLIM);
        }
    }
    for (int o = 16; o; o >>= 1) {
        my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
        bad_id |= __shfl_xor_sync(0xffffffffu, bad_id, o);
        bad_t |= __shfl_xor_sync(0xffffffffu, bad_t, o);
        loops += __shfl_xor_sync(0xffffffffu, loops, o);
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->max_id, my_max);
        if (bad_id) atomicOr(&st->bad_id, 1u);
        if (bad_t) atomicOr(&st->bad_t, 1u);
        if (loops) atomicAdd(&st->loops, loops);
        if (lo != LLONG_MAX) atomicMin(&st->tmin, lo);
        if (hi != LLONG_MIN) atomicMax(&st->tmax, hi);
    }
}

// The device address of page-locked host memory (cudaMallocHost,
// cudaHostAlloc, cudaHostRegister) allocated under the current device, which
// kernels read directly over the host link; nullptr for pageable memory, for
// another device's allocation, or when p is not aligned to `align` bytes.
const void *mapped_host(const void *p, size_t align) {
    if (!p || reinterpret_cast<uintptr_t>(p) % align) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // the failed query leaves a (non-sticky) error behind
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.device == dev ? a.devicePointer : nullptr;
}

// kept edges in input order: eidx = original index, tk = timestamp
__global__ void compact_kernel(const uint8_t *keep, const uint32_t *pos, size_t m, const int64_t *t,
                               uint32_t *eidx, int64_t *tk) {
    GRID_STRIDE(i, m) {
        if (keep[i]) {
            eidx[pos[i]] = (uint32_t)i;
            tk[pos[i]] = t[i];
        }
    }
}

__global__ void time_key_kernel(int64_t *tk, size_t m, int64_t tmin, uint64_t *tkey, uint32_t *vals,
                                const uint32_t *eidx) {
    GRID_STRIDE(i, m) {
        tkey[i] = (uint64_t)(tk[i] - tmin);
        vals[i] = eidx[i];
    }
}

// Packed key with the kept-edge index as tie-break (used when it fits in 63
// bits), and the pair key lo * n + hi as the value to carry.  eidx == nullptr:
// every input edge was kept (no self-loops), kept index = input index.
__global__ void key_direct_kernel(const uint32_t *eidx, const int64_t *tk, size_t m, int64_t tmin, int shift,
                                  const uint32_t *src, const uint32_t *dst, uint64_t n, uint64_t *key,
                                  uint64_t *pkey) {
    GRID_STRIDE(i, m) {
        const uint32_t e = eidx ? eidx[i] : (uint32_t)i;
        const uint32_t a = src[e], b = dst[e];
        key[i] = ((uint64_t)(tk[i] - tmin) << shift) | ((uint64_t)i << 1) | (uint64_t)(a > b);
        pkey[i] = (uint64_t)min(a, b) * n + max(a, b);
    }
}

__global__ void head_flags_kernel(const uint64_t *k, size_t m, uint8_t *head) {
    GRID_STRIDE(i, m) head[i] = (i == 0) || (k[i] != k[i - 1]);
}

__global__ void group_start_kernel(const uint8_t *head, const uint32_t *gid, size_t m, uint32_t *gstart) {
    GRID_STRIDE(i, m) if (head[i]) gstart[gid[i]] = (uint32_t)i;
}

__global__ void group_rank_max_kernel(const uint32_t *gid, const uint32_t *gstart, size_t m,
                                      unsigned int *max_rank) {
    unsigned int mx = 0;
    // gid is the exclusive scan of head flags, so element i's group is gid[i + 1] - 1
    GRID_STRIDE(i, m) mx = max(mx, (uint32_t)i - gstart[gid[i + 1] - 1]);
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(max_rank, mx);
}

// packed key and pair key per time-sorted edge
__global__ void pack_kernel(const uint64_t *tkey, const uint32_t *eidx, const uint32_t *gid,
                            const uint32_t *gstart, const uint32_t *src, const uint32_t *dst, size_t m, int shift,
                            uint64_t n, uint64_t *pkey, uint64_t *key) {
    GRID_STRIDE(i, m) {
        const uint32_t e = eidx[i];
        const uint32_t a = src[e], b = dst[e];
        const uint64_t rank = (uint32_t)i - gstart[gid[i + 1] - 1];
        const uint64_t dir = a > b;  // 1: from the larger id to the smaller
        key[i] = (tkey[i] << shift) | (rank << 1) | dir;
        const uint64_t lo = min(a, b), hi = max(a, b);
        pkey[i] = lo * n + hi;
    }
}

__global__ void pair_rle_kernel(const uint64_t *pkey, const uint8_t *head, const uint32_t *pid, size_t m,
                                uint64_t n, uint32_t *poff, uint2 *pair_vtx) {
    GRID_STRIDE(i, m) {
        if (head[i]) {
            const uint32_t p = pid[i];
            poff[p] = (uint32_t)i;
            pair_vtx[p] = make_uint2((uint32_t)(pkey[i] / n), (uint32_t)(pkey[i] % n));
        }
    }
}

__global__ void dir0_flags_kernel(const int64_t *key, size_t m, uint8_t *f) {
    GRID_STRIDE(i, m) f[i] = (key[i] & 1) == 0;
}

// Static degrees.  The pairs are sorted by (lo, hi), so the pairs of one
// lower endpoint u are the run [lo_first[u], lo_first[u] + lo_cnt[u]): its
// two ends are found where lo changes (plain stores, no atomics, even for a
// hub), and only the higher endpoints are counted with atomics (hi_cnt).
// Also the longest pair (sigma_max).
__global__ void pair_sizes_kernel(const uint32_t *poff, size_t ms, const uint2 *pv, uint32_t *lo_first,
                                  unsigned int *hi_cnt, unsigned int *sigma_max) {
    unsigned int mx = 0;
    GRID_STRIDE(p, ms) {
        mx = max(mx, poff[p + 1] - poff[p]);
        const uint2 e = pv[p];
        if (p == 0 || pv[p - 1].x != e.x) lo_first[e.x] = (uint32_t)p;
        atomicAdd(&hi_cnt[e.y], 1u);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(sigma_max, mx);
}

// deg = lo_cnt + hi_cnt, with lo_cnt written at each run's end.
__global__ void lo_runs_kernel(size_t ms, const uint2 *pv, const uint32_t *lo_first, unsigned int *lo_cnt) {
    GRID_STRIDE(p, ms) {
        const uint32_t x = pv[p].x;
        if (p + 1 == ms || pv[p + 1].x != x) lo_cnt[x] = (uint32_t)p + 1 - lo_first[x];
    }
}

__global__ void deg_sum_kernel(size_t n, const unsigned int *lo_cnt, const unsigned int *hi_cnt, unsigned int *deg) {
    GRID_STRIDE(v, n) deg[v] = lo_cnt[v] + hi_cnt[v];
}

// Adjacency lists: u's higher neighbours first, in pair order at fixed
// places (coalesced, no atomics), then its lower neighbours through a cursor
// (hi_cur, zeroed).
__global__ void adj_fill_kernel(const uint2 *pv, size_t ms, const uint32_t *adj_off, const uint32_t *lo_first,
                                const unsigned int *lo_cnt, unsigned int *hi_cur, uint32_t *adj) {
    GRID_STRIDE(p, ms) {
        const uint2 e = pv[p];
        adj[adj_off[e.x] + ((uint32_t)p - lo_first[e.x])] = e.y;
        adj[adj_off[e.y] + lo_cnt[e.y] + atomicAdd(&hi_cur[e.y], 1u)] = e.x;
    }
}


// ---------------------------------------------------------------- per-pair key sort
// After the pair sort each pair's edges are contiguous but in input order;
// these kernels sort every pair's keys in place (keys are unique, so the
// result does not depend on which unit sorts which pair).  Up to 8 edges:
// one thread, a sorting network in registers; up to 32: one warp, a bitonic
// network in registers; up to SEG_BIG_CAP: a warp or a CTA with up to 16
// keys per thread in registers (cross-warp stages through shared memory),
// one instance per power-of-two size class.
constexpr uint32_t SEG_BIG_CAP = 16384;  // largest pair sorted in place

// Pairs of 2..SEG_TINY_CAP edges: one thread, a sorting network in registers.
constexpr uint32_t SEG_TINY_CAP = 8;

__device__ __forceinline__ void cmp_swap(int64_t &a, int64_t &b) {
    const int64_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

__global__ void seg_sort_tiny_kernel(int64_t *key, const uint32_t *poff, uint32_t ms) {
    GRID_STRIDE(p, (size_t)ms) {
        const uint32_t b = poff[p], len = poff[p + 1] - b;
        if (len <= 1 || len > SEG_TINY_CAP) continue;
        int64_t x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = (uint32_t)j < len ? key[b + j] : INT64_MAX;
        // Batcher's odd-even merge sort network for 8 inputs (19 comparators)
        cmp_swap(x[0], x[1]); cmp_swap(x[2], x[3]); cmp_swap(x[4], x[5]); cmp_swap(x[6], x[7]);
        cmp_swap(x[0], x[2]); cmp_swap(x[1], x[3]); cmp_swap(x[4], x[6]); cmp_swap(x[5], x[7]);
        cmp_swap(x[1], x[2]); cmp_swap(x[5], x[6]);
        cmp_swap(x[0], x[4]); cmp_swap(x[1], x[5]); cmp_swap(x[2], x[6]); cmp_swap(x[3], x[7]);
        cmp_swap(x[2], x[4]); cmp_swap(x[3], x[5]);
        cmp_swap(x[1], x[2]); cmp_swap(x[3], x[4]); cmp_swap(x[5], x[6]);
#pragma unroll
        for (int j = 0; j < 8; j++)
            if ((uint32_t)j < len) key[b + j] = x[j];
    }
}

// Pairs of SEG_TINY_CAP+1..32 edges (listed in `small`): one warp, a bitonic
// network in registers.
// The list of a class is the slice [base[c], base[c] + count[c]) of `lists`
// (device memory, so no host round trip is needed).
__global__ void seg_sort_small_kernel(int64_t *key, const uint32_t *poff, const uint32_t *lists,
                                      const unsigned int *base, const unsigned int *count) {
    const uint32_t *small = lists + base[0];
    const uint32_t nsmall = count[0];
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nsmall;
         w += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t p = small[w], b = poff[p], len = poff[p + 1] - b;
        int64_t x = lane < len ? key[b + lane] : INT64_MAX;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const int64_t y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                x = keep_min ? min(x, y) : max(x, y);
            }
        }
        if (lane < len) key[b + lane] = x;
    }
}

// Size classes of the pairs above SEG_TINY_CAP edges: class 0 = 9..32 edges,
// class c = 1..9 = (2^(c+4), 2^(c+5)] edges, class 10 = longer than
// SEG_BIG_CAP (sorted together by radix sorts instead).
constexpr int SEG_CLASSES = 11;

__device__ __forceinline__ int seg_class(uint32_t len) {
    if (len <= SEG_TINY_CAP) return -1;
    if (len <= 32) return 0;
    if (len > SEG_BIG_CAP) return SEG_CLASSES - 1;
    return (32 - __clz(len - 1)) - 5;
}

// Per-class counts of the pairs (FILL = false), or each pair appended to its
// class's slice of `list` (FILL = true; `cursor` starts at the class
// offsets).  Warp-aggregated per class; the order inside a class is
// immaterial.
template <bool FILL>
__global__ void seg_classify_kernel(const uint32_t *poff, uint32_t ms, unsigned int *cursor, uint32_t *list) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t span = (ms + 31) & ~uint64_t(31);  // whole warps stay in the loop
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < span; p += stride) {
        const int c = p < ms ? seg_class(poff[p + 1] - poff[p]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        unsigned int base = 0;
        if (c >= 0 && (int)lane == leader) base = atomicAdd(&cursor[c], (unsigned int)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (FILL && c >= 0) list[base + __popc(peers & ((1u << lane) - 1))] = (uint32_t)p;
    }
}

// Pairs too long for the in-place sorts (nb of them, pair r listed in
// list[r]): their starts and lengths, for the long-pair sort below.
__global__ void long_pair_list_kernel(const uint32_t *list, uint32_t nb, const uint32_t *poff, uint32_t *start,
                                      uint64_t *len) {
    GRID_STRIDE(r, (size_t)nb) {
        const uint32_t p = list[r];
        start[r] = poff[p];
        len[r] = poff[p + 1] - poff[p];
    }
}

// Long pair of element j of their concatenation (pre: exclusive prefix of
// their lengths).
__device__ __forceinline__ uint32_t long_pair_of(const uint64_t *pre, uint32_t nb, uint64_t j) {
    uint32_t lo = 0, hi = nb;  // last r with pre[r] <= j
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

// The long pairs' keys are gathered with each pair's rank, sorted by key and
// then stably by rank, and written back into the same slots.
__global__ void long_pair_gather_kernel(const int64_t *key, const uint32_t *start, const uint64_t *pre, uint32_t nb,
                                        uint64_t total, uint64_t *gk, uint32_t *gr) {
    GRID_STRIDE(j, total) {
        const uint32_t r = long_pair_of(pre, nb, j);
        gk[j] = (uint64_t)key[start[r] + (j - pre[r])];
        gr[j] = r;
    }
}

__global__ void long_pair_rank_kernel(const uint32_t *gr, uint64_t total, uint64_t *rk) {
    GRID_STRIDE(j, total) rk[j] = gr[j];
}

__global__ void long_pair_scatter_kernel(const uint64_t *gk, const uint32_t *start, const uint64_t *pre, uint32_t nb,
                                         uint64_t total, int64_t *key) {
    GRID_STRIDE(j, total) {
        const uint32_t r = long_pair_of(pre, nb, j);
        key[start[r] + (j - pre[r])] = (int64_t)gk[j];
    }
}

// Class offsets in the list array (exclusive prefix of the counts) and the
// fill cursors; one thread.
__global__ void seg_bases_kernel(const unsigned int *count, unsigned int *base, unsigned int *cursor) {
    unsigned int run = 0;
    for (int c = 0; c < SEG_CLASSES; c++) {
        base[c] = run;
        cursor[c] = run;
        run += count[c];
    }
}

// Bitonic sort of T * E keys held by T consecutive threads, E per thread in
// registers (element i = t * E + r for thread t of the group).  A stage whose
// partner element sits in the same thread compares registers; a partner in
// another lane of the warp comes by shuffle; a partner in another warp (CTA
// groups only) is exchanged through shared memory s_x (r-major, so a warp's
// accesses are consecutive).
template <int E, int T>
__device__ __forceinline__ void bitonic_regs(int64_t (&x)[E], uint32_t t, int64_t *s_x) {
    constexpr uint32_t N = (uint32_t)E * T;
    for (uint32_t k = 2; k <= N; k <<= 1) {
        // stages whose partner is another thread (j >= E): same register r
        for (uint32_t j = k >> 1; j >= (uint32_t)E; j >>= 1) {
            const uint32_t tj = j / E;  // partner thread t ^ tj
            const bool lower = (t & tj) == 0;
            if (T <= 32 || tj < 32) {
#pragma unroll
                for (int r = 0; r < E; r++) {
                    const int64_t y = __shfl_xor_sync(0xffffffffu, x[r], tj);
                    const bool asc = ((t * E + r) & k) == 0;
                    x[r] = (lower == asc) ? min(x[r], y) : max(x[r], y);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; r++) s_x[r * T + t] = x[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < E; r++) {
                    const int64_t y = s_x[r * T + (t ^ tj)];
                    const bool asc = ((t * E + r) & k) == 0;
                    x[r] = (lower == asc) ? min(x[r], y) : max(x[r], y);
                }
                __syncthreads();
            }
        }
        // stages inside one thread's registers (j < E, j < k)
#pragma unroll
        for (int j = E / 2; j > 0; j >>= 1) {
            if ((uint32_t)j < k) {
#pragma unroll
                for (int r = 0; r < E; r++) {
                    if ((r & j) == 0) {
                        const int q = r | j;
                        const bool asc = ((t * E + r) & k) == 0;
                        const int64_t a = x[r], c = x[q];
                        const bool sw = (a > c) == asc;
                        x[r] = sw ? c : a;
                        x[q] = sw ? a : c;
                    }
                }
            }
        }
    }
}

// Sorts one pair's keys [b, b + len) with T threads holding E keys each
// (T * E >= len; the rest is padded with the largest key).
template <int E, int T>
__device__ __forceinline__ void sort_pair_regs(int64_t *key, uint32_t b, uint32_t len, uint32_t t, int64_t *s_x) {
    int64_t x[E];
#pragma unroll
    for (int r = 0; r < E; r++) {
        const uint32_t i = t * E + r;
        x[r] = i < len ? key[b + i] : INT64_MAX;
    }
    bitonic_regs<E, T>(x, t, s_x);
#pragma unroll
    for (int r = 0; r < E; r++) {
        const uint32_t i = t * E + r;
        if (i < len) key[b + i] = x[r];
    }
}

// One pair per group of T threads (a warp when T = 32, four groups per CTA;
// the whole CTA otherwise), E keys per thread: pairs of up to E * T edges.
template <int E, int T>
__global__ void __launch_bounds__(T >= 128 ? T : 128)
    seg_sort_group_kernel(int64_t *key, const uint32_t *poff, const uint32_t *lists, const unsigned int *base,
                          const unsigned int *count, int cls) {
    const uint32_t *list = lists + base[cls];
    const uint32_t nlist = count[cls];
    extern __shared__ int64_t s_x[];
    constexpr uint32_t CTA = T >= 128 ? T : 128, G = CTA / T;
    const uint32_t grp = threadIdx.x / T, t = threadIdx.x % T;
    for (uint64_t w = (uint64_t)blockIdx.x * G + grp; w < nlist; w += (uint64_t)gridDim.x * G) {
        const uint32_t p = list[w], b = poff[p], len = poff[p + 1] - b;
        sort_pair_regs<E, T>(key, b, len, t, s_x);
    }
}

// ---------------------------------------------------------------- k-core peel
// Counters of one phase of the peel.  Phases rotate through three slots: the
// slot of phase p is read by every thread after the barrier that ends p and
// is zeroed again after the barrier that ends p + 1, two barriers before it
// is written again.
struct PeelSlot {
    unsigned long long front;  // (vertices << 40) | their adjacency total
    unsigned int rem_n;
    int min_deg;
};
struct PeelCtl {
    PeelSlot slot[3];
    unsigned int kappa;
    unsigned int rounds;
    unsigned int error;
    unsigned int handoff;  // 1: stopped with at most tail_n vertices left
    int k;                 // level at the hand-off
    unsigned int rem_n;    // vertices left at the hand-off
    unsigned int rem_in_b; // the remaining list is in remB (else remA)
    unsigned int core_alive;  // vertices the cluster stage hands to one CTA
    // grid barrier of the grid-wide stage: the arrival counter and the
    // generation word sit on cache lines of their own, so the waiting CTAs'
    // polls do not queue behind the arrivals
    alignas(128) unsigned int bar_count;
    alignas(128) unsigned int bar_gen;
};

constexpr uint64_t MASK40 = (uint64_t(1) << 40) - 1;
constexpr int PEEL_THREADS = 1024;
constexpr int PEEL_RUN = 4;  // relaxed edges per thread per step
constexpr uint32_t PEEL_CACHE = 8192;  // frontier entries cached in shared memory
constexpr uint32_t CORE_PER_MAX = 8192;  // core vertices one CTA of the core cluster holds

// Frontier pushes of one CTA are staged in its shared memory and reach the
// global frontier with one device-memory atomic per CTA and phase (flush), so
// no counter in device memory is hit by every warp.  An entry is a vertex's
// adjacency start with its adjacency length; reservations are packed
// (entries << 40 | adjacency total).  A reservation that would overflow the
// stage goes straight to the global frontier instead.
constexpr uint32_t PEEL_STAGE = 4096;  // staged entries per CTA
constexpr size_t PEEL_SMEM = (size_t)(2 * PEEL_CACHE + 2 * PEEL_STAGE) * 4;  // dynamic shared memory

struct PeelStage {
    unsigned long long cnt;  // reserved in the stage (packed)
    unsigned long long cut;  // first reservation that did not fit (packed), or ~0
    unsigned long long gbase;
    unsigned long long total;
    unsigned int rem;        // compaction: kept vertices staged
    unsigned int rem_cut;    // compaction: first reservation that did not fit, or ~0
    unsigned int rem_gbase;
    unsigned int rem_total;
    int min_deg;
};

// Every lane of the warp must call it (pred selects the appending lanes).
__device__ __forceinline__ void push_frontier(bool pred, uint32_t ab, uint32_t nadj, PeelSlot *sl, uint32_t *front,
                                              uint32_t *foff, uint32_t lane, PeelStage *st, uint32_t *s_ab,
                                              uint32_t *s_off) {
    const uint64_t pk = pred ? ((uint64_t(1) << 40) | nadj) : 0;
    uint64_t x = pk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    const uint64_t tot = __shfl_sync(0xffffffffu, x, 31);
    if (!tot) return;
    uint64_t base = 0;
    int staged = 0;
    if (lane == 31) {
        base = atomicAdd(&st->cnt, (unsigned long long)tot);
        if ((base >> 40) + (tot >> 40) <= PEEL_STAGE) {
            staged = 1;
        } else {
            atomicMin(&st->cut, (unsigned long long)base);
            base = atomicAdd(&sl->front, (unsigned long long)tot);
        }
    }
    base = __shfl_sync(0xffffffffu, base, 31);
    staged = __shfl_sync(0xffffffffu, staged, 31);
    if (pred) {
        const uint64_t mine = base + x - pk;
        const uint32_t fi = (uint32_t)(mine >> 40);
        if (staged) {
            s_ab[fi] = ab;
            s_off[fi] = (uint32_t)(mine & MASK40);
        } else {
            front[fi] = ab;
            foff[fi] = (uint32_t)(mine & MASK40);
        }
    }
}

// Copies the CTA's staged frontier entries to the global frontier (one
// reservation) and resets the stage.  Every thread of the CTA calls it.
__device__ __forceinline__ void flush_frontier(PeelSlot *sl, uint32_t *front, uint32_t *foff, PeelStage *st,
                                               const uint32_t *s_ab, const uint32_t *s_off) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t = st->cnt < st->cut ? st->cnt : st->cut;
        st->total = t;
        st->gbase = t ? atomicAdd(&sl->front, t) : 0;
        st->cnt = 0;
        st->cut = ~0ull;
    }
    __syncthreads();
    const uint32_t n = (uint32_t)(st->total >> 40), fb = (uint32_t)(st->gbase >> 40);
    const uint32_t eb = (uint32_t)(st->gbase & MASK40);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        front[fb + i] = s_ab[i];
        foff[fb + i] = eb + s_off[i];
    }
}

// Last index fi in [0, fn) with foff[fi] <= x, for a non-decreasing foff
// with foff[0] = 0 <= x, by one warp (every lane calls it): each round the
// lanes probe 32 evenly spaced places and keep the stretch between the last
// one at or below x and the next, so fn offsets take about log32 fn
// dependent device-memory loads instead of log2 fn.
__device__ __forceinline__ uint32_t warp_last_le(const uint32_t *foff, uint32_t fn, uint32_t x, uint32_t lane) {
    uint32_t lo = 0, hi = fn;  // the answer is in [lo, hi); foff[lo] <= x
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t pos = lo + lane * step;
        const unsigned bal = __ballot_sync(0xffffffffu, pos < hi && __ldcg(foff + pos) <= x);
        lo += (31 - __clz(bal)) * step;  // lane 0 probes lo itself, so bal != 0
        hi = min(hi, lo + step);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, lo + lane < hi && __ldcg(foff + lo + lane) <= x);
    return lo + (31 - __clz(bal));
}

// Phase barrier of the grid-wide peel: every CTA of a cooperative launch,
// through an arrival counter and a generation word in device memory.  The
// wait is bounded; a CTA that gives up reports failure so the kernel stops.
constexpr uint32_t GRID_BAR_SPIN = 1u << 24;
constexpr unsigned GRID_BAR_SLEEP_NS = 32;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct GridSync {
    uint32_t gen = 0;
    __device__ uint32_t nthreads() const { return gridDim.x * blockDim.x; }
    __device__ uint32_t rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ bool sync(PeelCtl *ctl) {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            __threadfence();
            const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(&ctl->bar_count, 0u);
                __threadfence();
                atomicExch(&ctl->bar_gen, gen + 1);
            } else {
                uint32_t spins = 0;
                while (ld_acquire_gpu(&ctl->bar_gen) == gen) {
                    if (++spins > GRID_BAR_SPIN) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(GRID_BAR_SLEEP_NS);
                }
            }
            __threadfence();
            s_ok = ok;
        }
        gen++;
        __syncthreads();
        return s_ok != 0;
    }
};

// Level-synchronous bucketed peel (Sec. 3, degeneracy ordering).  At level k
// the frontier is every remaining vertex of degree <= k; removing it lowers
// its remaining neighbours' degrees, and a neighbour whose degree falls to k
// (the decrement that returns k + 1) joins the next round's frontier.  When a
// round empties the frontier, the remaining set is compacted and k rises to
// its smallest degree.  level[v] = round of removal; orienting every pair
// from the lower (round, id) to the higher gives each vertex at most k <=
// kappa out-neighbours.  This kernel runs the rounds on every SM while many
// vertices remain; it stops at the first level boundary with at most tail_n
// vertices left and records where it stopped in ctl, and peel_core_kernel
// peels the rest in one thread-block cluster.  Every control decision is
// uniform.
__global__ void __launch_bounds__(PEEL_THREADS)
    peel_kernel(const uint32_t *__restrict__ adj_off, const uint32_t *__restrict__ adj, int *deg,
                uint32_t *level, uint32_t *remA, uint32_t *remB, uint32_t *frontA, uint32_t *frontB,
                uint32_t *foffA, uint32_t *foffB, uint32_t n, uint32_t tail_n, PeelCtl *ctl) {
    GridSync bar;
    const uint32_t nthr = bar.nthreads();
    const uint32_t tid = bar.rank();
    const uint32_t lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    extern __shared__ uint32_t peel_smem[];
    uint32_t *s_foff = peel_smem, *s_front = peel_smem + PEEL_CACHE;
    uint32_t *s_ab = peel_smem + 2 * PEEL_CACHE, *s_off = s_ab + PEEL_STAGE;
    __shared__ PeelStage stg;
    __shared__ uint32_t s_slice[2];  // frontier slots of a CTA's first and last edge
    if (threadIdx.x == 0) {
        stg.cnt = 0;
        stg.cut = ~0ull;
        stg.rem = 0;
        stg.rem_cut = ~0u;
        stg.min_deg = INT_MAX;
    }
    __syncthreads();
    uint32_t *rem = remA, *rem_next = remB;
    uint32_t *front = frontA, *front_next = frontB, *foff = foffA, *foff_next = foffB;
    uint32_t rem_n = n, fn = 0, fe = 0;
    bool identity = true;  // the remaining set is 0..n-1 until the first compaction
    int k = 0;
    uint32_t round = 0, kappa = 0, ph = 0;
    bool stopped = false;  // handed the rest to the core stage
    const uint64_t ph_cap = 3ull * n + 8;
    bool ok = true;
    // ends phase ph: barrier, then zero the slot of phase ph + 2
    // (nullptr: a barrier gave up; the kernel stops at once)
    auto end_phase = [&]() -> PeelSlot * {
        if (!bar.sync(ctl)) {
            ok = false;
            return nullptr;
        }
        PeelSlot *cur = &ctl->slot[ph % 3];
        if (tid == 0) {
            PeelSlot *z = &ctl->slot[(ph + 2) % 3];
            z->front = 0;
            z->rem_n = 0;
            z->min_deg = INT_MAX;
        }
        ph++;
        if (ph > ph_cap) ok = false;
        return cur;
    };
    while (ok) {
        if (fn == 0) {
            // compaction: keep the unremoved vertices, find their smallest degree
            PeelSlot *sl = &ctl->slot[ph % 3];
            int my_min = INT_MAX;
            for (uint32_t base = 0; base < rem_n; base += nthr) {
                const uint32_t i = base + tid;
                uint32_t v = 0;
                bool keep = false;
                if (i < rem_n) {
                    v = identity ? i : __ldcg(rem + i);
                    keep = __ldcg(level + v) == UNSET;
                    if (keep) my_min = min(my_min, __ldcg(deg + v));
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                uint32_t b = 0;
                int staged = 0;
                if (lane == 0 && bal) {
                    const unsigned c = (unsigned)__popc(bal);
                    b = atomicAdd(&stg.rem, c);
                    if (b + c <= PEEL_STAGE) {
                        staged = 1;
                    } else {
                        atomicMin(&stg.rem_cut, b);
                        b = atomicAdd(&sl->rem_n, c);
                    }
                }
                b = __shfl_sync(0xffffffffu, b, 0);
                staged = __shfl_sync(0xffffffffu, staged, 0);
                if (keep) {
                    const uint32_t at = b + __popc(bal & lt_mask);
                    if (staged) s_ab[at] = v; else rem_next[at] = v;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) my_min = min(my_min, __shfl_xor_sync(0xffffffffu, my_min, o));
            if (lane == 0 && my_min != INT_MAX) atomicMin(&stg.min_deg, my_min);
            // one reservation and one minimum per CTA
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned t = min(stg.rem, stg.rem_cut);
                stg.rem_total = t;
                stg.rem_gbase = t ? atomicAdd(&sl->rem_n, t) : 0;
                if (stg.min_deg != INT_MAX) atomicMin(&sl->min_deg, stg.min_deg);
                stg.rem = 0;
                stg.rem_cut = ~0u;
                stg.min_deg = INT_MAX;
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < stg.rem_total; i += blockDim.x) rem_next[stg.rem_gbase + i] = s_ab[i];
            const PeelSlot *r = end_phase();
            if (!r) break;
            rem_n = __ldcg(&r->rem_n);
            const int md = __ldcg(&r->min_deg);
            identity = false;
            uint32_t *t = rem; rem = rem_next; rem_next = t;
            if (rem_n == 0) break;
            k = max(k, md);
            if (rem_n <= tail_n) {  // hand the rest to the core stage
                if (tid == 0) {
                    ctl->handoff = 1;
                    ctl->k = k;
                    ctl->rem_n = rem_n;
                    ctl->rem_in_b = rem == remB;
                }
                stopped = true;
                break;
            }
            kappa = max(kappa, (uint32_t)k);
            // collection: the new level's frontier
            sl = &ctl->slot[ph % 3];
            for (uint32_t base = 0; base < rem_n; base += nthr) {
                const uint32_t i = base + tid;
                bool take = false;
                uint32_t v = 0, na = 0;
                uint32_t ab = 0;
                if (i < rem_n) {
                    v = __ldcg(rem + i);
                    take = __ldcg(deg + v) <= k;
                    if (take) {
                        level[v] = round;
                        ab = adj_off[v];
                        na = adj_off[v + 1] - ab;
                    }
                }
                push_frontier(take, ab, na, sl, front, foff, lane, &stg, s_ab, s_off);
            }
            flush_frontier(sl, front, foff, &stg, s_ab, s_off);
            r = end_phase();
            if (!r) break;
            const uint64_t f = __ldcg(&r->front);
            fn = (uint32_t)(f >> 40);
            fe = (uint32_t)(f & MASK40);
        }
        // relaxation: remove the frontier (round `round`).  The round's
        // edges are dealt to the CTAs in equal contiguous ranges (every SM
        // takes part however small the round), a CTA stages the slice of the
        // frontier that covers its range in shared memory (two warp-parallel
        // searches of the offsets), and each thread takes PEEL_RUN
        // consecutive edges, finds their vertex in the slice and issues
        // their loads and atomics as independent batches.
        PeelSlot *sl = &ctl->slot[ph % 3];
        const uint32_t cper = (fe + gridDim.x - 1) / gridDim.x;
        const uint32_t cb = min(fe, blockIdx.x * cper), ce = min(fe, cb + cper);
        for (uint32_t sb = cb; sb < ce; sb += blockDim.x * PEEL_RUN) {  // uniform per CTA
            const uint32_t se = min(ce, sb + blockDim.x * PEEL_RUN);
            if (threadIdx.x < 64) {
                const uint32_t fi = warp_last_le(foff, fn, threadIdx.x < 32 ? sb : se - 1, lane);
                if (lane == 0) s_slice[threadIdx.x >> 5] = fi;
            }
            __syncthreads();
            const uint32_t f0 = s_slice[0], nsl = s_slice[1] - f0 + 1;
            const bool cached = nsl <= PEEL_CACHE;
            if (cached)
                for (uint32_t i = threadIdx.x; i < nsl; i += blockDim.x) {
                    s_foff[i] = __ldcg(foff + f0 + i);
                    s_front[i] = __ldcg(front + f0 + i);
                }
            __syncthreads();
            const uint32_t fb = cached ? f0 : 0u, fc = cached ? nsl : fn;  // the slice searched
            auto ld_foff = [&](uint32_t i) { return cached ? s_foff[i] : __ldcg(foff + i); };
            auto ld_front = [&](uint32_t i) { return cached ? s_front[i] : __ldcg(front + i); };
            const uint32_t e0 = sb + threadIdx.x * PEEL_RUN;
            uint32_t wv[PEEL_RUN];
            bool live[PEEL_RUN];
            if (e0 < se) {
                uint32_t lo = 0, hi = fc;  // last slot of the slice with offset <= e0
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (ld_foff(mid) <= e0) lo = mid; else hi = mid;
                }
                uint32_t fi = lo;
                uint32_t fbeg = ld_foff(fi);
                uint32_t fend = fb + fi + 1 < fn ? (fi + 1 < fc ? ld_foff(fi + 1) : __ldcg(foff + fb + fi + 1)) : fe;
                uint32_t base = ld_front(fi);
#pragma unroll
                for (int j = 0; j < PEEL_RUN; j++) {
                    const uint32_t e = e0 + j;
                    live[j] = e < se;
                    if (live[j]) {
                        while (e >= fend) {  // the next vertex (inside the slice: e < se)
                            fi++;
                            fbeg = fend;
                            fend = fb + fi + 1 < fn ? (fi + 1 < fc ? ld_foff(fi + 1) : __ldcg(foff + fb + fi + 1)) : fe;
                            base = ld_front(fi);
                        }
                        wv[j] = adj[base + (e - fbeg)];
                    }
                }
                // no level check: a removed vertex already has degree <= k,
                // so a decrement returns k + 1 only for a remaining vertex
            } else {
#pragma unroll
                for (int j = 0; j < PEEL_RUN; j++) live[j] = false;
            }
            int old[PEEL_RUN];
#pragma unroll
            for (int j = 0; j < PEEL_RUN; j++) old[j] = live[j] ? atomicSub(deg + wv[j], 1) : 0;
#pragma unroll
            for (int j = 0; j < PEEL_RUN; j++) {
                const bool push = live[j] && old[j] == k + 1;
                uint32_t na = 0, ab = 0;
                if (push) {
                    level[wv[j]] = round + 1;
                    ab = adj_off[wv[j]];
                    na = adj_off[wv[j] + 1] - ab;
                }
                push_frontier(push, ab, na, sl, front_next, foff_next, lane, &stg, s_ab, s_off);
            }
            __syncthreads();  // the slice is read before the next one is staged
        }
        flush_frontier(sl, front_next, foff_next, &stg, s_ab, s_off);
        const PeelSlot *r = end_phase();
        if (!r) break;
        const uint64_t f = __ldcg(&r->front);
        fn = (uint32_t)(f >> 40);
        fe = (uint32_t)(f & MASK40);
        round++;
        uint32_t *t = front; front = front_next; front_next = t;
        t = foff; foff = foff_next; foff_next = t;
    }
    if (tid == 0) {
        ctl->rounds = round;
        ctl->kappa = kappa;
        if (!stopped) ctl->handoff = 0;
        if (!ok) ctl->error = 1;
    }
}



// ---------------------------------------------------------------- peel core
// The last (cluster size x CORE_PER_MAX) or fewer vertices are peeled by one
// thread-block cluster that keeps every remaining vertex's state in
// distributed shared memory.  Their adjacency among themselves is first
// rebuilt with local ids.

// Local ids of the remaining vertices and their (current) degrees.
__global__ void tail_ids_kernel(const uint32_t *rem, uint32_t R, const int *deg, uint32_t *lid, uint32_t *cdeg) {
    GRID_STRIDE(i, (size_t)R) {
        lid[rem[i]] = (uint32_t)i;
        cdeg[i] = (uint32_t)deg[rem[i]];
    }
}

// Adjacency of the remaining vertices among themselves, in local ids.  The
// full adjacency lists of the remaining vertices are cut into chunks of
// TAIL_CHUNK entries (chunk_pre: exclusive prefix of chunks per vertex); one
// CTA takes one chunk and appends the remaining neighbours to the vertex's
// slice through a per-vertex cursor (order inside a slice is immaterial).
constexpr uint32_t TAIL_CHUNK = 4096;

__global__ void tail_chunks_kernel(const uint32_t *rem, uint32_t R, const uint32_t *adj_off, uint32_t *nchunk) {
    GRID_STRIDE(i, (size_t)R) {
        const uint32_t v = rem[i];
        nchunk[i] = (adj_off[v + 1] - adj_off[v] + TAIL_CHUNK - 1) / TAIL_CHUNK;
    }
}

__global__ void __launch_bounds__(256)
    tail_adj_kernel(const uint32_t *rem, uint32_t R, const uint32_t *chunk_pre, const uint32_t *adj_off,
                    const uint32_t *adj, const uint32_t *level, const uint32_t *lid, const uint32_t *coff,
                    uint32_t *cursor, uint32_t *cadj) {
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_base;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t nchunks = chunk_pre[R];
    for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        uint32_t lo = 0, hi = R;  // vertex of chunk c: last i with chunk_pre[i] <= c
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (chunk_pre[mid] <= c) lo = mid; else hi = mid;
        }
        const uint32_t i = lo, v = rem[i];
        const uint32_t b = adj_off[v] + (c - chunk_pre[i]) * TAIL_CHUNK;
        const uint32_t e = min(adj_off[v + 1], b + TAIL_CHUNK);
        for (uint32_t j0 = b; j0 < e; j0 += 256) {
            const uint32_t j = j0 + threadIdx.x;
            bool keep = false;
            uint32_t x = 0;
            if (j < e) {
                x = adj[j];
                keep = level[x] == UNSET;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_w[w] = __popc(bal);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t run = 0;
                for (int k = 0; k < 8; k++) {
                    const uint32_t t = s_w[k];
                    s_w[k] = run;
                    run += t;
                }
                s_base = run ? atomicAdd(cursor + i, run) : 0;
            }
            __syncthreads();
            if (keep) cadj[coff[i] + s_base + s_w[w] + __popc(bal & lt_mask)] = lid[x];
            __syncthreads();
        }
    }
}

// The peel of the core (Sec. 3, same level-synchronous rule as peel_kernel)
// in one thread-block cluster.  Local vertex l is owned by CTA l / per, which
// holds its remaining degree, level, adjacency span and, when it is in a
// frontier, its frontier entry, all in shared memory.  A round: each CTA
// relaxes the edges of its own frontier vertices (adjacency read from L2);
// level checks and degree decrements go to the owner's shared memory
// (distributed shared memory); a vertex whose degree falls to k joins its
// owner's next frontier.  Only counts cross the cluster barrier: pushes are
// tallied per CTA in a slot that rotates over three rounds, so a slot is
// read by every CTA between the barriers that end round r and r + 1 and is
// zeroed in round r + 2.  Continues from level ctl->k and round
// ctl->rounds; writes level[] of the core vertices it removes and hands the
// last (at most stop_n) to peel_tail_kernel.
constexpr int CORE_THREADS = 1024;      // per CTA of the cluster (measured: more threads per round beat fewer idle warps)
constexpr int CORE_TAIL_THREADS = 1024;  // the one-CTA run of the last PEEL_TAIL vertices
constexpr uint32_t PEEL_TAIL = 8192;     // the cluster hands the last this many to one CTA
constexpr int CORE_RUN = 8;          // adjacency entries a lane relaxes per step (measured: 8 beat 4)
constexpr uint32_t CORE_MAX_CLUSTER = 16;

// degree, adjacency start, adjacency length, two frontier buffers and the
// level of `per` owned vertices (u32 each)
inline size_t core_smem_bytes(uint32_t per) { return (size_t)per * 6 * 4; }

// `per` (a power of two) vertices per CTA.
__global__ void __launch_bounds__(CORE_THREADS, 1)
    peel_core_kernel(const uint32_t *rem, uint32_t R, uint32_t per, const uint32_t *coff, const uint32_t *cadj,
                     uint32_t *level, int *deg, uint32_t stop_n, uint32_t *alive_out, PeelCtl *ctl) {
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t crank = cl.block_rank(), csize = cl.num_blocks();
    const uint32_t per_lg = (uint32_t)(__ffs(per) - 1);
    // shared memory of the CTA that owns a vertex
    auto at = [&](auto *p, uint32_t own) { return cl.map_shared_rank(p, own); };
    auto csync = [&]() { cl.sync(); };
    const uint32_t tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
    extern __shared__ __align__(16) uint32_t core_smem[];
    uint32_t *s_deg = core_smem, *s_ab = s_deg + per, *s_na = s_ab + per;
    uint32_t *s_front = s_na + per;  // [2][per]
    uint32_t *s_lev = s_front + 2 * per;
    __shared__ unsigned int s_fcnt[2];                 // entries in my frontier buffers, by round parity
    __shared__ unsigned int s_tot[3];                  // the cluster's pushes, per round mod 3
    __shared__ unsigned int s_peer[2];                 // this CTA's pushes, by round parity
    __shared__ int s_mins[CORE_MAX_CLUSTER];           // each CTA's smallest remaining degree
    __shared__ unsigned int s_alive[CORE_MAX_CLUSTER]; // and its number of remaining vertices
    __shared__ unsigned int s_nalive;
    __shared__ int s_min;
    const uint32_t base_lid = crank * per;
    const uint32_t my_n = R > base_lid ? min(per, R - base_lid) : 0;
    for (uint32_t i = tid; i < my_n; i += nthr) {
        const uint32_t ab = coff[base_lid + i], na = coff[base_lid + i + 1] - ab;
        s_ab[i] = ab;
        s_na[i] = na;
        s_deg[i] = na;
        s_lev[i] = UNSET;
    }
    if (tid == 0) {
        s_fcnt[0] = s_fcnt[1] = 0;
        s_tot[0] = s_tot[1] = s_tot[2] = 0;
        s_peer[0] = s_peer[1] = 0;
        s_min = INT_MAX;
        s_nalive = 0;
    }
    int k = __ldcg(&ctl->k);
    const uint32_t round0 = __ldcg(&ctl->rounds);
    uint32_t kappa = __ldcg(&ctl->kappa);
    uint32_t round = 0, cur = 0;
    bool need_level = true, ok = true, stopped = false;
    csync();  // every CTA's state is initialised before any remote access
    for (;;) {
        if (need_level) {
            // new level: the cluster's smallest remaining degree, then every
            // owned vertex of degree <= k joins this CTA's frontier
            int my = INT_MAX;
            unsigned int na = 0;
            for (uint32_t i = tid; i < my_n; i += nthr)
                if (s_lev[i] == UNSET) {
                    my = min(my, (int)s_deg[i]);
                    na++;
                }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                my = min(my, __shfl_xor_sync(0xffffffffu, my, o));
                na += __shfl_xor_sync(0xffffffffu, na, o);
            }
            if (lane == 0 && my != INT_MAX) atomicMin(&s_min, my);
            if (lane == 0 && na) atomicAdd(&s_nalive, na);
            __syncthreads();
            if (tid < csize) {
                at(s_mins, tid)[crank] = s_min;
                at(s_alive, tid)[crank] = s_nalive;
            }
            csync();
            int g = lane < csize ? s_mins[lane] : INT_MAX;
            unsigned int alive = lane < csize ? s_alive[lane] : 0u;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                g = min(g, __shfl_xor_sync(0xffffffffu, g, o));
                alive += __shfl_xor_sync(0xffffffffu, alive, o);
            }
            if (tid == 0) s_nalive = 0;  // read above; next written after a later barrier
            if (g == INT_MAX) break;  // nothing left anywhere (uniform)
            if (alive <= stop_n) {
                // hand the rest to one CTA: its vertices (ids) and their
                // current degrees; levels of the removed ones below
                for (uint32_t i = tid; i < my_n; i += nthr) {
                    if (s_lev[i] == UNSET) {
                        const uint32_t v = rem[base_lid + i];
                        alive_out[atomicAdd(&ctl->core_alive, 1u)] = v;
                        deg[v] = (int)s_deg[i];
                    }
                }
                if (crank == 0 && tid == 0) {
                    ctl->k = max(k, g);
                    ctl->rem_n = alive;
                }
                stopped = true;
                break;
            }
            k = max(k, g);
            kappa = max(kappa, (uint32_t)k);
            for (uint32_t i = tid; i < my_n; i += nthr) {
                if (s_lev[i] == UNSET && (int)s_deg[i] <= k) {
                    s_lev[i] = round;
                    s_front[cur * per + atomicAdd(&s_fcnt[cur], 1u)] = i;
                }
            }
            // every CTA has collected before any CTA decrements its
            // neighbours' degrees (else a vertex a slow CTA is still
            // collecting could also be pushed)
            csync();
            if (tid == 0) s_min = INT_MAX;
            need_level = false;
        }
        // relaxation of this CTA's frontier (round `round`)
        const uint32_t nxt = cur ^ 1, slot = round % 3;
        const uint32_t fn = s_fcnt[cur];
        const uint32_t *F = s_front + cur * per;
        const uint32_t par = round & 1;
        // the tally slot of round - 2: every CTA read it before the barrier
        // that ended round - 1
        if (tid == 0) s_tot[(round + 1) % 3] = 0;
        // one warp per frontier vertex, its lanes over the adjacency,
        // CORE_RUN entries a lane per step with their loads in flight together
        const uint32_t wid = tid >> 5, nwarp = nthr >> 5;
        for (uint32_t fi = wid; fi < fn; fi += nwarp) {
            const uint32_t fv = F[fi], ab = s_ab[fv], na = s_na[fv];
            for (uint32_t j0 = 0; j0 < na; j0 += 32 * CORE_RUN) {
                uint32_t wv[CORE_RUN];
                bool live[CORE_RUN];
#pragma unroll
                for (int j = 0; j < CORE_RUN; j++) {
                    const uint32_t e = j0 + (uint32_t)j * 32 + lane;
                    live[j] = e < na;
                    wv[j] = live[j] ? cadj[ab + e] : 0u;
                }
                // no level check: a removed vertex already has degree <= k, so
                // a decrement can return k + 1 only for a remaining vertex, once
                uint32_t own[CORE_RUN], idx[CORE_RUN];
#pragma unroll
                for (int j = 0; j < CORE_RUN; j++) {
                    own[j] = live[j] ? wv[j] >> per_lg : 0u;
                    idx[j] = live[j] ? wv[j] & (per - 1) : 0u;
                }
                uint32_t old[CORE_RUN];
#pragma unroll
                for (int j = 0; j < CORE_RUN; j++)
                    old[j] = live[j] ? atomicSub(at(s_deg, own[j]) + idx[j], 1u) : 0;
#pragma unroll
                for (int j = 0; j < CORE_RUN; j++) {
                    if (live[j] && (int)old[j] == k + 1) {
                        at(s_lev, own[j])[idx[j]] = round + 1;
                        const uint32_t slot_at = atomicAdd(at(s_fcnt, own[j]) + nxt, 1u);
                        at(s_front, own[j])[nxt * per + slot_at] = idx[j];
                        atomicAdd(&s_peer[par], 1u);
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_fcnt[cur] = 0;  // consumed; others push into it only after the barrier
        // add this CTA's pushes to every CTA's tally of this round before
        // the barrier, so that after it each CTA reads the total locally
        if (tid < csize && s_peer[par]) atomicAdd(at(s_tot, tid) + slot, s_peer[par]);
        cl.sync();
        const uint32_t pushed = s_tot[slot];
        // read above, before this barrier; counted into again two rounds on
        if (tid == 0) s_peer[par] = 0;
        round++;
        cur = nxt;
        need_level = pushed == 0;
        if (round > R + 1) {  // cannot happen: every round removes a vertex
            ok = false;
            break;
        }
    }
    for (uint32_t i = tid; i < my_n; i += nthr)
        if (s_lev[i] != UNSET) level[rem[base_lid + i]] = round0 + s_lev[i];
    if (crank == 0 && tid == 0) {
        ctl->rounds = round0 + round;
        ctl->kappa = kappa;
        ctl->handoff = stopped ? 1u : 0u;
        if (!ok) ctl->error = 1;
    }
    csync();  // no CTA leaves while another may still read its shared memory
}

// The last R <= PEEL_TAIL vertices, peeled by one CTA (Sec. 3, the same
// level-synchronous rule).  Shared memory holds each vertex's remaining
// degree, level and adjacency start (coff, R + 1 entries), and two frontier
// buffers of (vertex, offset of its first chunk among the round's chunks),
// where a chunk is PEEL_CHUNK consecutive adjacency entries of one vertex.
// A push reserves its frontier slot and its chunks with one packed 64-bit
// shared-memory add ((vertices << 40) | chunks), so the offsets are an
// exclusive prefix of the chunk counts in slot order.  A round deals the
// frontier's chunks to the warps (chunk c to warp c mod 32; its vertex by a
// warp-uniform binary search over the offsets), so a hub in the frontier is
// spread over many warps instead of stepping through its list on one, and a
// round costs about one dependent L2 load.  The round's packed counts rotate
// over three slots (read in round r, pushed into in round r - 1, zeroed in
// round r + 1, which starts after the barrier that ends r), so a round ends
// on one barrier.  The per-vertex arrays are padded to a multiple of four
// and scanned with 16-byte shared-memory loads at each new level.
constexpr uint32_t PEEL_CHUNK = 32 * CORE_RUN;

__host__ __device__ inline uint32_t tail_pad(uint32_t R) { return (R + 3) & ~3u; }
// degree, level, coff (+4), two u32 offset buffers, two u16 vertex buffers
inline size_t tail_smem_bytes(uint32_t R) { return ((size_t)6 * tail_pad(R) + 4) * 4; }

// Warp-collective (every lane calls it): lane appends its vertices v[j] with
// bit j of pm set (chunk counts ch[j]) to the frontier whose packed count is
// *pk, in j order.
template <int N>
__device__ __forceinline__ void tail_push(uint32_t pm, const uint32_t (&v)[N], const uint32_t (&ch)[N],
                                          unsigned long long *pk, uint16_t *fv, uint32_t *fo, uint32_t lane) {
    const unsigned bal = __ballot_sync(0xffffffffu, pm != 0);
    if (!bal) return;
    uint64_t own = (uint64_t)__popc(pm) << 40;
#pragma unroll
    for (int j = 0; j < N; j++)
        if (pm >> j & 1) own += ch[j];
    uint64_t mine;
    if (__popc(bal) == 1) {
        if (!pm) return;
        mine = atomicAdd(pk, (unsigned long long)own);
    } else {
        uint64_t x = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        uint64_t base = 0;
        if (lane == 31) base = atomicAdd(pk, (unsigned long long)x);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (!pm) return;
        mine = base + x - own;
    }
    uint32_t fi = (uint32_t)(mine >> 40), off = (uint32_t)(mine & MASK40);
#pragma unroll
    for (int j = 0; j < N; j++)
        if (pm >> j & 1) {
            fv[fi] = (uint16_t)v[j];
            fo[fi] = off;
            fi++;
            off += ch[j];
        }
}

__device__ __forceinline__ uint32_t tail_chunks(const uint32_t *s_coff, uint32_t v) {
    return (s_coff[v + 1] - s_coff[v] + PEEL_CHUNK - 1) / PEEL_CHUNK;
}

__global__ void __launch_bounds__(CORE_TAIL_THREADS, 1)
    peel_tail_kernel(const uint32_t *rem, uint32_t R, const uint32_t *coff, const uint32_t *cadj,
                     uint32_t *level, PeelCtl *ctl) {
    extern __shared__ __align__(16) uint32_t tail_smem[];
    const uint32_t Rp = tail_pad(R);
    uint32_t *s_deg = tail_smem, *s_lev = s_deg + Rp, *s_coff = s_lev + Rp;  // s_coff: R + 1 used
    uint32_t *s_fo = s_coff + Rp + 4;                                        // [2][Rp] chunk offsets
    uint16_t *s_fv = reinterpret_cast<uint16_t *>(s_fo + 2 * Rp);            // [2][Rp] vertices
    __shared__ unsigned long long s_fpack[3];
    __shared__ int s_min;
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x, nwarp = nthr >> 5;
    // s_coff[i] for i >= R is coff[R] (padding vertices have no entries);
    // each entry has one writer
    for (uint32_t i = tid; i <= Rp; i += nthr) {
        const uint32_t c = coff[min(i, R)];
        s_coff[i] = c;
        if (i < Rp) {
            s_deg[i] = i < R ? coff[i + 1] - c : 0u;
            s_lev[i] = i < R ? UNSET : 0u;  // padding counts as removed
        }
    }
    if (tid == 0) {
        s_fpack[0] = s_fpack[1] = s_fpack[2] = 0;
        s_min = INT_MAX;
    }
    int k = __ldcg(&ctl->k);
    const uint32_t round0 = __ldcg(&ctl->rounds);
    uint32_t kappa = __ldcg(&ctl->kappa);
    uint32_t round = 0;
    bool need_level = true, ok = true;
    const uint4 *deg4 = reinterpret_cast<const uint4 *>(s_deg), *lev4 = reinterpret_cast<const uint4 *>(s_lev);
    __syncthreads();
    for (;;) {
        const uint32_t slot = round % 3, buf = round & 1;
        if (need_level) {
            // new level: the smallest remaining degree, then every remaining
            // vertex of degree <= k joins this round's frontier
            int my = INT_MAX;
            for (uint32_t i4 = tid; i4 < Rp / 4; i4 += nthr) {
                const uint4 d = deg4[i4], l = lev4[i4];
                if (l.x == UNSET) my = min(my, (int)d.x);
                if (l.y == UNSET) my = min(my, (int)d.y);
                if (l.z == UNSET) my = min(my, (int)d.z);
                if (l.w == UNSET) my = min(my, (int)d.w);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) my = min(my, __shfl_xor_sync(0xffffffffu, my, o));
            if (lane == 0 && my != INT_MAX) atomicMin(&s_min, my);
            __syncthreads();
            const int g = s_min;
            if (g == INT_MAX) break;  // nothing left (uniform)
            k = max(k, g);
            kappa = max(kappa, (uint32_t)k);
            for (uint32_t b0 = 0; b0 < Rp / 4; b0 += nthr) {  // uniform trip count: the push is warp-collective
                const uint32_t i4 = b0 + tid;
                uint32_t v[4], ch[4], pm = 0;
                if (i4 < Rp / 4) {
                    const uint4 d = deg4[i4], l = lev4[i4];
                    const uint32_t dd[4] = {d.x, d.y, d.z, d.w}, ll[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        v[c] = 4 * i4 + c;
                        ch[c] = 0;
                        if (ll[c] == UNSET && (int)dd[c] <= k) {
                            s_lev[v[c]] = round;
                            ch[c] = tail_chunks(s_coff, v[c]);
                            pm |= 1u << c;
                        }
                    }
                }
                tail_push(pm, v, ch, &s_fpack[slot], s_fv + buf * Rp, s_fo + buf * Rp, lane);
            }
            __syncthreads();
            if (tid == 0) s_min = INT_MAX;  // every thread read it before the barrier above
            need_level = false;
        }
        // relaxation of round `round`: chunk c belongs to the last frontier
        // slot whose offset is <= c
        const unsigned long long fp = s_fpack[slot];
        const uint32_t fn = (uint32_t)(fp >> 40), nch = (uint32_t)(fp & MASK40);
        if (tid == 0) s_fpack[(round + 2) % 3] = 0;  // read in round - 1, pushed into in round + 1
        const uint16_t *FV = s_fv + buf * Rp;
        const uint32_t *FO = s_fo + buf * Rp;
        uint16_t *NV = s_fv + (buf ^ 1) * Rp;
        uint32_t *NO = s_fo + (buf ^ 1) * Rp;
        unsigned long long *npk = &s_fpack[(round + 1) % 3];
        for (uint32_t c = wid; c < nch; c += nwarp) {  // warp-uniform
            uint32_t lo = 0, hi = fn;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (FO[mid] <= c) lo = mid; else hi = mid;
            }
            const uint32_t fv = FV[lo], ab = s_coff[fv], na = s_coff[fv + 1] - ab;
            const uint32_t e0 = (c - FO[lo]) * PEEL_CHUNK;
            uint32_t w[CORE_RUN];
            bool live[CORE_RUN];
#pragma unroll
            for (int j = 0; j < CORE_RUN; j++) {
                const uint32_t e = e0 + (uint32_t)j * 32 + lane;
                live[j] = e < na;
                w[j] = live[j] ? cadj[ab + e] : 0u;
            }
            // no level check: a removed vertex already has degree <= k, so
            // a decrement returns k + 1 only for a remaining vertex, once
            uint32_t old[CORE_RUN];
#pragma unroll
            for (int j = 0; j < CORE_RUN; j++) old[j] = live[j] ? atomicSub(s_deg + w[j], 1u) : 0u;
            uint32_t pch[CORE_RUN], pm = 0;
#pragma unroll
            for (int j = 0; j < CORE_RUN; j++) {
                pch[j] = 0;
                if (live[j] && (int)old[j] == k + 1) {
                    s_lev[w[j]] = round + 1;
                    pch[j] = tail_chunks(s_coff, w[j]);
                    pm |= 1u << j;
                }
            }
            tail_push(pm, w, pch, npk, NV, NO, lane);
        }
        __syncthreads();
        const bool pushed = *npk != 0;
        round++;
        need_level = !pushed;
        if (round > R + 1) {  // cannot happen: every round removes a vertex
            ok = false;
            break;
        }
    }
    for (uint32_t i = tid; i < R; i += nthr)
        if (s_lev[i] != UNSET) level[rem[i]] = round0 + s_lev[i];
    if (tid == 0) {
        ctl->rounds = round0 + round;
        ctl->kappa = kappa;
        ctl->handoff = 0;
        if (!ok) ctl->error = 1;
    }
}

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
    // splitmix64 finaliser, used only to draw a random vertex order
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)(x ^ (x >> 31));
}

// Ordering key of each vertex (ties by id come from the stable sort of the
// identity permutation): its peel level, degree, a hash, or nothing (id).
__global__ void order_key_kernel(uint32_t n, uint32_t orientation, const uint32_t *level, const unsigned int *deg,
                                 uint64_t seed, uint64_t *hi_out, uint32_t *ident, unsigned int *hi_max) {
    unsigned int mx = 0;
    GRID_STRIDE(v, (size_t)n) {
        uint32_t hi;
        switch (orientation) {
            case TTC_ORIENT_ID: hi = 0; break;
            case TTC_ORIENT_DEGREE: hi = deg[v]; break;
            case TTC_ORIENT_RANDOM: hi = mix32(seed ^ (v * 0x100000001b3ull)); break;
            default: hi = level[v]; break;
        }
        hi_out[v] = hi;
        ident[v] = (uint32_t)v;
        mx = max(mx, hi);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(hi_max, mx);
}

__global__ void rank_scatter_kernel(const uint32_t *id_of, uint32_t n, uint32_t *rank_of) {
    GRID_STRIDE(r, (size_t)n) rank_of[id_of[r]] = (uint32_t)r;
}

// Orients each static edge from the lower to the higher rank; the key
// (source rank, target rank) sorts the out-lists by target rank.
__global__ void orient_kernel(const uint2 *pv, size_t ms, const uint32_t *rank_of, uint64_t n, uint64_t *okey,
                              uint32_t *oval) {
    GRID_STRIDE(p, ms) {
        const uint32_t ra = rank_of[pv[p].x], rb = rank_of[pv[p].y];
        const uint32_t s = ra < rb ? ra : rb, d = ra < rb ? rb : ra;
        okey[p] = (uint64_t)s * n + d;
        oval[p] = (uint32_t)p;
    }
}

// CSR offsets from sorted keys: off[r] = #{i : keys[i] < r * mult} for
// r = 0..nv (binary search per r).
__global__ void offsets_from_sorted_kernel(const uint64_t *keys, size_t len, uint64_t mult, uint32_t nv,
                                           uint32_t *off) {
    GRID_STRIDE(r, (size_t)nv + 1) {
        const uint64_t x = (uint64_t)r * mult;
        size_t lo = 0, cnt = len;
        while (cnt > 0) {
            const size_t half = cnt >> 1;
            if (keys[lo + half] < x) {
                lo += half + 1;
                cnt -= half + 1;
            } else {
                cnt = half;
            }
        }
        off[r] = (uint32_t)lo;
    }
}

// Largest gap between consecutive offsets (the largest list).
__global__ void max_gap_kernel(const uint32_t *off, size_t nv, unsigned int *mx_out) {
    unsigned int mx = 0;
    GRID_STRIDE(i, nv) mx = max(mx, off[i + 1] - off[i]);
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(mx_out, mx);
}

// Splits the sorted keys into source and target ranks and sets up the sort
// of the oriented edges by target (key = target rank, value = position).
__global__ void split_okey_kernel(const uint64_t *okey, size_t ms, uint64_t n, uint32_t *osrc, uint32_t *onbr,
                                  uint64_t *tkey, uint32_t *tpos) {
    GRID_STRIDE(i, ms) {
        const uint32_t d = (uint32_t)(okey[i] % n);
        osrc[i] = (uint32_t)(okey[i] / n);
        onbr[i] = d;
        tkey[i] = d;
        tpos[i] = (uint32_t)i;
    }
}

__global__ void widen_kernel(const uint32_t *a, const uint32_t *b, size_t n, uint64_t *a64, uint64_t *b64) {
    GRID_STRIDE(i, n) {
        a64[i] = a[i];
        b64[i] = b[i];
    }
}

// ---------------------------------------------------------------- triangles
struct RecCtx {
    uint32_t labeling;
    uint64_t light_max;
};

// Per oriented edge a -> b (rank order): its pair's multiplicity σ (capped at
// 2^31 - 1; a cap only moves a triangle between two exact counting bins) and,
// in bit 31, whether id(a) > id(b).
constexpr uint32_t SIG_MASK = 0x7fffffffu;

// ocsr[i] = (target rank, sigma word, pair id, 0) of oriented edge i, so one
// 16-byte load gives the enumeration everything it needs about an edge.
__global__ void osig_kernel(const uint32_t *opair, const uint32_t *osrc, const uint32_t *onbr, const uint32_t *id_of,
                            const uint32_t *poff, size_t ms, uint4 *ocsr) {
    GRID_STRIDE(i, ms) {
        const uint32_t p = opair[i], sig = poff[p + 1] - poff[p], b = onbr[i];
        const uint32_t down = id_of[osrc[i]] > id_of[b] ? 0x80000000u : 0u;
        ocsr[i] = make_uint4(b, (sig < SIG_MASK ? sig : SIG_MASK) | down, p, 0u);
    }
}

// Names the triangle's vertices u, v, w for counting and returns the record.
// The triangle was found as u0 < v0 < w0 in the ordering with oriented edges
// u0 -> v0, u0 -> w0, v0 -> w0: pairs p_*, packed (σ, id order) words s_*.
// The flip bits say, per record pair, whether the labelled direction runs
// from the larger id to the smaller.
__device__ __forceinline__ uint4 make_record(const RecCtx &c, uint32_t s_uv, uint32_t s_uw, uint32_t s_vw,
                                             uint32_t p_uv, uint32_t p_uw, uint32_t p_vw, bool *heavy,
                                             uint32_t *n_a = nullptr, uint32_t *n_b = nullptr) {
    const uint32_t n_uv = s_uv & SIG_MASK, n_uw = s_uw & SIG_MASK, n_vw = s_vw & SIG_MASK;
    const bool g_uv = s_uv >> 31, g_uw = s_uw >> 31, g_vw = s_vw >> 31;  // id(u0) > id(v0), ...
    uint32_t A = p_uv, B = p_uw, C = p_vw, nA = n_uv, nB = n_uw;
    bool fa = g_uv, fb = g_uw, fc = g_vw;  // (U, V, W) = (u0, v0, w0)
    if (c.labeling == TTC_LABEL_HEAVIEST_VW) {
        if (n_uw > n_vw && n_uw >= n_uv) {  // {u0, w0} is only searched: (U, V, W) = (v0, u0, w0)
            A = p_uv; B = p_vw; C = p_uw; nA = n_uv; nB = n_vw;
            fa = !g_uv; fb = g_vw; fc = g_uw;
        } else if (n_uv > n_vw && n_uv > n_uw) {  // {u0, v0}: (U, V, W) = (w0, u0, v0)
            A = p_uw; B = p_vw; C = p_uv; nA = n_uw; nB = n_vw;
            fa = !g_uw; fb = !g_vw; fc = g_uv;
        }
    }
    *heavy = (uint64_t)nA * nB >= c.light_max;
    if (n_a) *n_a = nA;
    if (n_b) *n_b = nB;
    const uint32_t flags = (fa ? TriRec::FLIP_A : 0u) | (fb ? TriRec::FLIP_B : 0u) | (fc ? TriRec::FLIP_C : 0u);
    return make_uint4(A, B, C, flags);
}

// enumerated edges (sigma_A + sigma_B) of each heavy record
__global__ void heavy_sizes_kernel(const uint4 *rec, size_t nh, const uint32_t *poff, uint64_t *heavy_e) {
    GRID_STRIDE(i, nh) {
        const uint4 r = rec[i];
        heavy_e[i] = (uint64_t)(poff[r.x + 1] - poff[r.x]) + (poff[r.y + 1] - poff[r.y]);
    }
}

// sizes of heavy records and the work statistics of all records, from the
// records themselves (used when the enumeration's sigma words were capped)
__global__ void record_stats_kernel(const uint4 *rec, size_t tau, uint64_t n_light, const uint32_t *poff,
                                    uint64_t *heavy_e, unsigned long long *sums) {
    unsigned long long w = 0, en = 0, wh = 0, lp = 0;
    GRID_STRIDE(i, tau) {
        const uint4 r = rec[i];
        const uint64_t a = poff[r.x + 1] - poff[r.x], b = poff[r.y + 1] - poff[r.y], c = poff[r.z + 1] - poff[r.z];
        w += 8 * (a + b + c) + 12;
        en += a + b;
        if (i >= n_light) {
            heavy_e[i - n_light] = a + b;
            wh += 8 * (a + b + c) + 12;
        } else {
            lp += a * b;
        }
    }
    for (int o = 16; o; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        en += __shfl_xor_sync(0xffffffffu, en, o);
        wh += __shfl_xor_sync(0xffffffffu, wh, o);
        lp += __shfl_xor_sync(0xffffffffu, lp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, w);
        atomicAdd(sums + 1, en);
        atomicAdd(sums + 2, wh);
        atomicAdd(sums + 3, lp);
    }
}

// Triangle enumeration (Sec. 5: each triangle is found once, from its
// oriented edges u -> v, u -> w, v -> w with u < v < w in the ordering).
// Vertices are named by rank and every out-list is sorted by rank, so for an
// in-edge u -> v at position e of N+(u), the candidates w are the suffix of
// N+(u) after e.  Work items are (v, 32 in-edges of v): the warp stages N+(v)
// in its shared memory (when it fits), flattens the 32 suffixes across its
// lanes, and each lane looks its element w up in N+(v) by binary search.
// One pass: the suffix length bounds an edge's triangles, so every oriented
// edge has that much room reserved in a scratch array (`resv`, an exclusive
// prefix of the suffix lengths); its light records fill the room from the
// front and its heavy records from the back, each at its rank among that
// edge's hits of that bin (hits of one edge come in ascending w), and the
// per-edge counts go to cnt_light / cnt_heavy.  tri_compact_kernel then
// copies every edge's records to their bins: the layout is deterministic.
constexpr int TRI_THREADS = 256;
constexpr int TRI_WARPS = TRI_THREADS / 32;
constexpr uint32_t TRI_NV_CAP = 448;  // most staged N+(v) entries per warp (4 CTAs per SM)

// Items: chunk c of target v covers its in-edges [32 c, 32 c + 32); a vertex
// with no out-edge closes no triangle as the middle vertex.
__global__ void tri_items_count_kernel(const uint32_t *out_off, const uint32_t *in_off, uint32_t n,
                                       uint32_t *nitems) {
    GRID_STRIDE(v, (size_t)n) {
        const uint32_t dout = out_off[v + 1] - out_off[v], din = in_off[v + 1] - in_off[v];
        nitems[v] = dout ? (din + 31) / 32 : 0;
    }
}

// One thread per item: its vertex is the last v with item_pre[v] <= c.
__global__ void tri_items_fill_kernel(const uint32_t *item_pre, uint32_t n, uint32_t nitems, uint2 *items) {
    GRID_STRIDE(c, (size_t)nitems) {
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_pre[mid] <= c) lo = mid; else hi = mid;
        }
        items[c] = make_uint2(lo, ((uint32_t)c - item_pre[lo]) * 32);
    }
}

struct TriCsr {
    const uint32_t *onbr;     // out-lists: target ranks, sorted
    const uint4 *ocsr;        // per oriented edge: target rank, (σ, id order) word, pair id
    const uint32_t *out_off;  // out-list offsets by rank
    const uint32_t *osrc;     // source rank of each oriented edge
    const uint32_t *in_off;   // in-list offsets by rank
    const uint32_t *in_e;     // in-lists: positions of the oriented edges
};

// Shared memory of one warp: N+(v) (target ranks, σ words and, when writing,
// pair ids) for dv <= TRI_NV_CAP.
constexpr size_t tri_warp_smem(uint32_t cap) { return (size_t)cap * 4 * 3; }
// Entries staged per warp: the largest out-degree rounded up to a warp, at
// most TRI_NV_CAP.  Shared memory the staging does not need stays L1 cache,
// which the dependent loads of the enumeration use (measured on the power-law
// workload, max out-degree 294: 320 entries 4.8 ms, 448 entries 5.2 ms).
inline uint32_t tri_nv_cap(uint64_t max_out_degree) {
    return (uint32_t)std::min<uint64_t>(TRI_NV_CAP, std::max<uint64_t>(32, (max_out_degree + 31) / 32 * 32));
}

// What an enumeration pass does with the triangles it finds.
enum EnumMode {
    ENUM_WRITE = 0,    // write every record into its edge's room (cnt_light/heavy, resv, sparse)
    ENUM_SCAN = 1,     // statistics and light/heavy totals; heavy records appended to `heavy`
    ENUM_COLLECT = 2,  // light records appended to `light` (streamed handle, one chunk of items)
};

struct EnumArgs {
    // ENUM_WRITE
    uint32_t *cnt_light, *cnt_heavy;
    const uint64_t *resv;
    uint4 *sparse;
    // ENUM_WRITE, ENUM_SCAN: sums[0..4] as below, ENUM_SCAN also sums[5..6] =
    // light, heavy triangles
    unsigned long long *sums;
    // ENUM_SCAN: heavy records, appended while heavy_n < heavy_cap
    uint4 *heavy;
    unsigned long long *heavy_n;
    uint64_t heavy_cap;
    // ENUM_COLLECT: light records, appended while light_n < light_cap
    uint4 *light;
    unsigned long long *light_n;
    uint64_t light_cap;
};

template <int EM>
__global__ void __launch_bounds__(TRI_THREADS)
    tri_enum_kernel(const uint2 *__restrict__ items, uint32_t nitems, TriCsr g, RecCtx rc, EnumArgs ea,
                    uint32_t nv_cap) {
    // work statistics of the records written: sum of 8 (s_A + s_B + s_C) + 12,
    // of s_A + s_B, the first over heavy records, of s_A s_B over light
    // ones, and whether a sigma word was capped
    unsigned long long st_w = 0, st_en = 0, st_wh = 0, st_lp = 0, st_cap = 0, st_nl = 0, st_nh = 0;
    extern __shared__ uint32_t tri_smem[];
    __shared__ uint32_t s_excl[TRI_WARPS][33];
    __shared__ uint32_t s_e[TRI_WARPS][32], s_se[TRI_WARPS][32], s_pe[TRI_WARPS][32];
    __shared__ uint64_t s_lo[TRI_WARPS][32], s_ho[TRI_WARPS][32];  // each slot's room: front, back
    __shared__ uint32_t s_run[TRI_WARPS][64];  // per in-edge slot: light, heavy hits so far
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t *s_nv = tri_smem + (size_t)w * (tri_warp_smem(nv_cap) / 4);
    uint32_t *s_nvs = s_nv + nv_cap, *s_nvp = s_nvs + nv_cap;
    uint32_t staged_v = 0xffffffffu;
    for (uint64_t it = (uint64_t)blockIdx.x * TRI_WARPS + w; it < nitems; it += (uint64_t)gridDim.x * TRI_WARPS) {
        const uint2 item = items[it];
        const uint32_t v = item.x, c0 = item.y;
        const uint32_t vb = __ldg(g.out_off + v), dv = __ldg(g.out_off + v + 1) - vb;
        const bool staged = dv <= nv_cap;
        if (staged && staged_v != v) {
            __syncwarp();
            for (uint32_t i = lane; i < dv; i += 32) {
                const uint4 q = __ldg(g.ocsr + vb + i);
                s_nv[i] = q.x;
                s_nvs[i] = q.y;
                s_nvp[i] = q.z;
            }
            staged_v = v;
        }
        __syncwarp();
        const uint32_t *nv = staged ? s_nv : g.onbr + vb;
        const uint32_t ib = __ldg(g.in_off + v), din = __ldg(g.in_off + v + 1) - ib;
        const uint32_t i = c0 + lane;
        uint32_t len = 0;
        if (i < din) {
            const uint32_t e = __ldg(g.in_e + ib + i), u = __ldg(g.osrc + e);
            const uint4 q = __ldg(g.ocsr + e);
            s_e[w][lane] = e;
            s_se[w][lane] = q.y;
            s_pe[w][lane] = q.z;
            len = __ldg(g.out_off + u + 1) - e - 1;  // the suffix of N+(u) after v
            if constexpr (EM == ENUM_WRITE) {
                s_lo[w][lane] = ea.resv[e];
                s_ho[w][lane] = ea.resv[e] + len - 1;
            }
        }
        s_run[w][2 * lane] = 0;
        s_run[w][2 * lane + 1] = 0;
        uint32_t x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        s_excl[w][lane] = x - len;
        const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
        if (lane == 0) s_excl[w][32] = total;
        __syncwarp();
        // two elements per lane per step (j and j + 32), their loads and
        // searches interleaved; ranks are then taken in element order
        const uint32_t top = dv ? 1u << (31 - __clz(dv)) : 0u;  // largest power of two <= dv
        for (uint32_t base = 0; base < total; base += 64) {
            uint32_t jj[2] = {base + lane, base + 32 + lane};
            uint32_t o[2] = {0, 0}, lo[2] = {0, 0};
            uint4 qw[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};  // the edge u -> w
            bool in[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                in[h] = jj[h] < total;
                if (in[h]) {
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (s_excl[w][o[h] + step] <= jj[h]) o[h] += step;
                    qw[h] = __ldg(g.ocsr + s_e[w][o[h]] + 1 + (jj[h] - s_excl[w][o[h]]));
                }
            }
            const uint32_t x3[2] = {qw[0].x, qw[1].x};
            // lower bound of x3 in N+(v), branch-free, both searches in step
            for (uint32_t step = top; step; step >>= 1) {
#pragma unroll
                for (int h = 0; h < 2; h++)
                    if (lo[h] + step <= dv && nv[lo[h] + step - 1] < x3[h]) lo[h] += step;
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                bool hit = false, heavy = false;
                uint4 r = make_uint4(0, 0, 0, 0);
                if (in[h] && lo[h] < dv && nv[lo[h]] == x3[h]) {
                    hit = true;
                    uint32_t s_vw, p_vw;  // the edge v -> w
                    if (staged) {
                        s_vw = s_nvs[lo[h]];
                        p_vw = s_nvp[lo[h]];
                    } else {
                        const uint4 q = __ldg(g.ocsr + vb + lo[h]);
                        s_vw = q.y;
                        p_vw = q.z;
                    }
                    uint32_t na, nb;
                    r = make_record(rc, s_se[w][o[h]], qw[h].y, s_vw, s_pe[w][o[h]], qw[h].z, p_vw, &heavy, &na,
                                    &nb);
                    if constexpr (EM != ENUM_COLLECT) {
                        const uint32_t s1 = s_se[w][o[h]] & SIG_MASK, s2 = qw[h].y & SIG_MASK,
                                       s3 = s_vw & SIG_MASK;
                        const unsigned long long wb = 8ull * ((unsigned long long)s1 + s2 + s3) + 12;
                        st_w += wb;
                        st_en += (unsigned long long)na + nb;
                        if (heavy) st_wh += wb; else st_lp += (unsigned long long)na * nb;
                        st_cap |= (s1 == SIG_MASK || s2 == SIG_MASK || s3 == SIG_MASK) ? 1ull : 0ull;
                    }
                    if constexpr (EM == ENUM_SCAN) {
                        if (heavy) {
                            st_nh++;
                            const unsigned long long at = atomicAdd(ea.heavy_n, 1ull);
                            if (at < ea.heavy_cap) ea.heavy[at] = r;
                        } else {
                            st_nl++;
                        }
                    }
                }
                if constexpr (EM == ENUM_COLLECT) {
                    // one reservation per warp for its light hits
                    const bool take = hit && !heavy;
                    const unsigned lm = __ballot_sync(0xffffffffu, take);
                    if (!lm) continue;
                    unsigned long long at = 0;
                    if (lane == (uint32_t)(__ffs(lm) - 1)) at = atomicAdd(ea.light_n, (unsigned long long)__popc(lm));
                    at = __shfl_sync(0xffffffffu, at, __ffs(lm) - 1) + __popc(lm & lt_mask);
                    if (take && at < ea.light_cap) ea.light[at] = r;
                }
                if constexpr (EM != ENUM_WRITE) continue;
                const unsigned act = __ballot_sync(0xffffffffu, hit);
                if (!act) continue;
                const uint32_t slot = o[h];
                const uint32_t key = slot * 2 + (heavy ? 1u : 0u);
                const unsigned peers = __match_any_sync(0xffffffffu, hit ? key : 0xffffffffu) & act;
                uint32_t rank = 0;
                if (hit) rank = s_run[w][key] + __popc(peers & lt_mask);
                __syncwarp();
                if (hit && (peers & lt_mask) == 0) s_run[w][key] += __popc(peers);
                __syncwarp();
                if (hit) ea.sparse[heavy ? s_ho[w][slot] - rank : s_lo[w][slot] + rank] = r;
            }
        }
        __syncwarp();
        if constexpr (EM == ENUM_WRITE) {
            if (i < din) {
                ea.cnt_light[s_e[w][lane]] = s_run[w][2 * lane];
                ea.cnt_heavy[s_e[w][lane]] = s_run[w][2 * lane + 1];
            }
        }
        __syncwarp();
    }
    if constexpr (EM == ENUM_COLLECT) {
        return;
    } else {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            st_w += __shfl_xor_sync(0xffffffffu, st_w, o);
            st_en += __shfl_xor_sync(0xffffffffu, st_en, o);
            st_wh += __shfl_xor_sync(0xffffffffu, st_wh, o);
            st_lp += __shfl_xor_sync(0xffffffffu, st_lp, o);
            st_cap |= __shfl_xor_sync(0xffffffffu, st_cap, o);
            st_nl += __shfl_xor_sync(0xffffffffu, st_nl, o);
            st_nh += __shfl_xor_sync(0xffffffffu, st_nh, o);
        }
        if (lane == 0 && st_w) {
            atomicAdd(ea.sums, st_w);
            atomicAdd(ea.sums + 1, st_en);
            atomicAdd(ea.sums + 2, st_wh);
            atomicAdd(ea.sums + 3, st_lp);
            if (st_cap) atomicOr(ea.sums + 4, 1ull);
            if constexpr (EM == ENUM_SCAN) {
                atomicAdd(ea.sums + 5, st_nl);
                atomicAdd(ea.sums + 6, st_nh);
            }
        }
    }
}


// Room reserved per oriented edge e = u -> v: the length of N+(u) after v.
__global__ void tri_room_kernel(const uint32_t *osrc, const uint32_t *out_off, size_t ms, uint64_t *room) {
    GRID_STRIDE(e, ms) room[e] = out_off[osrc[e] + 1] - (uint32_t)e - 1;
}

// Copies each oriented edge's records from its reserved room to the bins:
// light record r of edge e to light_off[e] + r, heavy record r (stored from
// the back of the room) to heavy_base + heavy_off[e] + r.  A warp takes 32
// consecutive edges and flattens their records over its lanes, so reads and
// writes run along contiguous ranges.
__global__ void __launch_bounds__(TRI_THREADS)
    tri_compact_kernel(const uint64_t *resv, const uint32_t *cnt_light, const uint32_t *cnt_heavy,
                       const uint64_t *light_off, const uint64_t *heavy_off, uint64_t heavy_base, size_t ms,
                       const uint4 *__restrict__ sparse, uint4 *__restrict__ tri) {
    __shared__ uint32_t s_excl[TRI_WARPS][33];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * TRI_WARPS;
    for (uint64_t e0 = ((uint64_t)blockIdx.x * TRI_WARPS + w) * 32; e0 < ms; e0 += nwarps * 32) {
        const uint64_t e = e0 + lane;
        for (int heavy = 0; heavy < 2; heavy++) {
            const uint32_t c = e < ms ? (heavy ? cnt_heavy[e] : cnt_light[e]) : 0;
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
            if (!total) continue;  // warp-uniform
            s_excl[w][lane] = x - c;
            if (lane == 0) s_excl[w][32] = total;
            __syncwarp();
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t j = base + lane;
                if (j < total) {
                    uint32_t o = 0;
#pragma unroll
                    for (uint32_t step = 16; step; step >>= 1)
                        if (s_excl[w][o + step] <= j) o += step;
                    const uint64_t eo = e0 + o;
                    const uint32_t r = j - s_excl[w][o];
                    if (heavy) tri[heavy_base + heavy_off[eo] + r] = sparse[resv[eo + 1] - 1 - r];
                    else tri[light_off[eo] + r] = sparse[resv[eo] + r];
                }
            }
            __syncwarp();
        }
    }
}

// Heavy-bin class of each heavy record from its enumerated size: 0 = one
// warp, 1 = one CTA, 2 = huge (flat path).
__global__ void heavy_class_kernel(const uint64_t *he, size_t nh, uint32_t wcap, uint32_t ccap, uint8_t *f0,
                                   uint8_t *f1, uint8_t *f2) {
    GRID_STRIDE(i, nh) {
        const uint64_t e = he[i];
        f0[i] = e <= wcap;
        f1[i] = e > wcap && e <= ccap;
        f2[i] = e > ccap;
    }
}

// Stable three-way partition of the heavy records (and their sizes).
__global__ void heavy_partition_kernel(const uint4 *rec, const uint64_t *he, const uint8_t *f0, const uint8_t *f1,
                                       const uint32_t *p0, const uint32_t *p1, const uint32_t *p2, size_t nh,
                                       uint64_t n0, uint64_t n1, uint4 *out, uint64_t *he_out) {
    GRID_STRIDE(i, nh) {
        const uint64_t dst = f0[i] ? p0[i] : f1[i] ? n0 + p1[i] : n0 + n1 + p2[i];
        out[dst] = rec[i];
        he_out[dst] = he[i];
    }
}

// A second stream forked from `main` (it waits for everything enqueued on
// main so far); fork_done() marks the end of its work, join() makes main wait
// for it.  Buffers allocated on it are released before it is destroyed
// (declare them after the SideStream).
struct SideStream {
    cudaStream_t s = nullptr, main;
    cudaEvent_t fork = nullptr, done = nullptr;
    explicit SideStream(cudaStream_t m) : main(m) {
        TTC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        TTC_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        TTC_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        TTC_CUDA(cudaEventRecord(fork, main));
        TTC_CUDA(cudaStreamWaitEvent(s, fork, 0));
    }
    SideStream(const SideStream &) = delete;
    SideStream &operator=(const SideStream &) = delete;
    void fork_done() { TTC_CUDA(cudaEventRecord(done, s)); }
    void join() { TTC_CUDA(cudaStreamWaitEvent(main, done, 0)); }
    ~SideStream() {
        cudaStreamSynchronize(s);
        cudaEventDestroy(fork);
        cudaEventDestroy(done);
        cudaStreamDestroy(s);
    }
};

template <typename T>
T read_scalar(const T *dev, cudaStream_t s) {
    T h;
    TTC_CUDA(cudaMemcpyAsync(&h, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

uint32_t default_light_max_pairs() { return 65; }

// The graph as a one-entry graph table for the count kernels.
// Records an enumeration work item (target v, in-edges c0 .. c0 + 31) can
// produce at most: the suffixes of N+(u) after v over its in-edges u -> v.
__global__ void item_room_kernel(const uint2 *items, uint32_t nitems, TriCsr g, uint64_t *room) {
    GRID_STRIDE(it, (size_t)nitems) {
        const uint2 item = items[it];
        const uint32_t ib = g.in_off[item.x], din = g.in_off[item.x + 1] - ib;
        uint64_t r = 0;
        for (uint32_t i = item.y; i < din && i < item.y + 32; i++) {
            const uint32_t e = g.in_e[ib + i];
            r += g.out_off[g.osrc[e] + 1] - e - 1;
        }
        room[it] = r;
    }
}

// After a collecting pass: the chunk's view lists its n light records, and
// its 32-record chunk prefix is {0, ceil(n / 32)}.
__global__ void chunk_view_kernel(const unsigned long long *light_n, uint64_t cap, GraphView *view,
                                  uint64_t *pre) {
    const uint64_t n = min((uint64_t)*light_n, cap);
    view->n_light = n;
    pre[0] = 0;
    pre[1] = (n + 31) / 32;
}

// One enumeration pass over the work items (grid: as many CTAs as fit),
// staging out-lists of up to nv_cap entries per warp.
template <int EM>
void launch_enum(const uint2 *items, uint32_t nitems, const TriCsr &tc, const RecCtx &rc, const EnumArgs &ea,
                 uint32_t nv_cap, cudaStream_t s) {
    if (!nitems) return;
    const size_t smem = TRI_WARPS * tri_warp_smem(nv_cap);
    ensure_smem((const void *)tri_enum_kernel<EM>, TRI_WARPS * tri_warp_smem(TRI_NV_CAP));
    int occ = 1;
    TTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tri_enum_kernel<EM>, TRI_THREADS, smem));
    const unsigned grid = (unsigned)std::min<uint64_t>(nitems / TRI_WARPS + 1, (uint64_t)sm_count() * std::max(1, occ));
    tri_enum_kernel<EM><<<grid, TRI_THREADS, smem, s>>>(items, nitems, tc, rc, ea, nv_cap);
    TTC_LAUNCH_CHECK();
}

static void set_view(ttc_graph *g, cudaStream_t s) {
    GraphView &v = g->view_host;
    v.key = g->key.get();
    v.fwd = g->fwd.get();
    v.poff = g->poff.get();
    v.tri = g->tri.get();
    v.n_light = g->streamed ? 0 : g->st.tau_light;  // a streamed handle lists heavy triangles only
    v.n_hwarp = g->st.tau_hwarp;
    v.n_hcta = g->st.tau_hcta;
    v.n_heavy = g->st.tau_heavy;
    v.span = g->span;
    v.shift = g->shift;
    v.wide = g->heavy_wide;
    v.strict = g->strict ? 1 : 0;
    v.m = g->st.m;
    v.ms = g->st.m_s;
    g->view.alloc(1, s);
    g->prefix.alloc(6, s);
    const uint64_t pre[6] = {0, (v.n_light + 31) / 32, 0, v.n_hwarp, 0, v.n_hcta};
    TTC_CUDA(cudaMemcpyAsync(g->view.get(), &v, sizeof v, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemcpyAsync(g->prefix.get(), pre, sizeof pre, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaStreamSynchronize(s));
}

// Largest cluster (up to 16 CTAs of 1024 threads) the device can run for the peel.
// CTAs of the grid-wide peel stage: all co-resident (cooperative launch),
// 0 when cooperative launches are unavailable.
int peel_grid_ctas() {
    static int ctas = -1;
    if (ctas >= 0) return ctas;
    int dev = 0, coop = 0, per_sm = 0;
    ctas = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ctas;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaFuncSetAttribute(peel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PEEL_SMEM);
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peel_kernel, PEEL_THREADS,
                                                              PEEL_SMEM) == cudaSuccess)
        ctas = std::max(0, per_sm) * sm_count();
    cudaGetLastError();
    return ctas;
}

// Cluster size for the core peel: 16 CTAs when such a cluster fits, else 8;
// -1 when neither does.
int core_cluster_size() {
    static int best = 0;
    if (best) return best;
    best = -1;
    cudaFuncSetAttribute(peel_core_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (cudaFuncSetAttribute(peel_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tail_smem_bytes(PEEL_TAIL)) != cudaSuccess ||
        cudaFuncSetAttribute(peel_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)core_smem_bytes(CORE_PER_MAX)) != cudaSuccess) {
        cudaGetLastError();
        return best;
    }
    for (int c = (int)CORE_MAX_CLUSTER; c >= 8; c /= 2) {
        const size_t smem = core_smem_bytes(CORE_PER_MAX);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(CORE_THREADS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, peel_core_kernel, &cfg) == cudaSuccess && clusters >= 1) {
            best = c;
            break;
        }
        cudaGetLastError();
    }
    return best;
}

// Launches the in-place sort of size class c with a grid that fills the GPU;
// the class's pair count is read on the device, so an empty class costs one
// short launch.
template <int E, int T>
void launch_seg_group(int64_t *key, const uint32_t *poff, const uint32_t *lists, const unsigned int *base,
                      const unsigned int *count, int c, cudaStream_t s) {
    constexpr int CTA = T >= 128 ? T : 128;
    const size_t smem = T >= 64 ? (size_t)E * T * 8 : 0;
    if (smem > 48 * 1024) ensure_smem((const void *)seg_sort_group_kernel<E, T>, smem);
    int occ = 0;
    TTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, seg_sort_group_kernel<E, T>, CTA, smem));
    const unsigned grid = (uint32_t)sm_count() * std::max(1, occ);
    seg_sort_group_kernel<E, T><<<grid, CTA, smem, s>>>(key, poff, lists, base, count, c);
    TTC_LAUNCH_CHECK();
}

void seg_sort_classes(int64_t *key, const uint32_t *poff, const uint32_t *lists, const unsigned int *base,
                      const unsigned int *count, cudaStream_t s) {
    seg_sort_small_kernel<<<(unsigned)sm_count() * 8, TPB, 0, s>>>(key, poff, lists, base, count);  // ..32
    TTC_LAUNCH_CHECK();
    launch_seg_group<2, 32>(key, poff, lists, base, count, 1, s);     // 33..64
    launch_seg_group<4, 32>(key, poff, lists, base, count, 2, s);     // ..128
    launch_seg_group<8, 32>(key, poff, lists, base, count, 3, s);     // ..256
    launch_seg_group<16, 32>(key, poff, lists, base, count, 4, s);    // ..512
    launch_seg_group<8, 128>(key, poff, lists, base, count, 5, s);    // ..1024
    launch_seg_group<4, 512>(key, poff, lists, base, count, 6, s);    // ..2048
    launch_seg_group<8, 512>(key, poff, lists, base, count, 7, s);    // ..4096
    launch_seg_group<16, 512>(key, poff, lists, base, count, 8, s);   // ..8192
    launch_seg_group<32, 512>(key, poff, lists, base, count, 9, s);   // ..16384
}

void build_graph(ttc_graph *g, const uint32_t *src_in, const uint32_t *dst_in, const int64_t *t_in, uint64_t m_in,
                 const LoadOptions &opt) {
    cudaStream_t s = g->stream;
    ttc_graph_stats &st = g->st;
    g->labeling = opt.labeling;
    // the light path decodes a pair's index within its triangle in float
    // arithmetic, exact below 2^20 pairs per triangle
    g->strict = (opt.flags & TTC_LOAD_STRICT_TIME) != 0;
    g->light_max_pairs = opt.light_max_pairs ? std::min<uint32_t>(opt.light_max_pairs, 1u << 20)
                                             : default_light_max_pairs();
    if (opt.orientation > TTC_ORIENT_RANDOM) fail(TTC_ERR_INVALID, "unknown orientation %u", opt.orientation);
    if (opt.labeling > TTC_LABEL_SOURCE) fail(TTC_ERR_INVALID, "unknown labeling %u", opt.labeling);
    if (m_in >= (uint64_t(1) << 32) - 1) fail(TTC_ERR_RANGE, "m = %llu exceeds 2^32 - 2 edges", (unsigned long long)m_in);
    const size_t m0 = (size_t)m_in;

    prof_begin(g, s, "load:ingest");
    // ---- a1: inputs on the device, validated
    DevBuf<uint32_t> src_buf, dst_buf;
    DevBuf<int64_t> t_buf;
    const uint32_t *src = src_in, *dst = dst_in;
    const int64_t *t = t_in;
    // what the ingest kernel reads, and where it writes the device copies
    // (page-locked host input only)
    const uint32_t *in_src = src_in, *in_dst = dst_in;
    const int64_t *in_t = t_in;
    uint32_t *copy_src = nullptr, *copy_dst = nullptr;
    int64_t *copy_t = nullptr;
    if (!(opt.flags & TTC_LOAD_DEVICE_INPUT) && m0) {
        src_buf.alloc(m0, s); dst_buf.alloc(m0, s); t_buf.alloc(m0, s);
        const void *hs = mapped_host(src_in, 4);
        const void *hd = mapped_host(dst_in, 4);
        const void *ht = mapped_host(t_in, 8);
        if (hs && hd && ht) {
            in_src = static_cast<const uint32_t *>(hs);
            in_dst = static_cast<const uint32_t *>(hd);
            in_t = static_cast<const int64_t *>(ht);
            copy_src = src_buf.get(); copy_dst = dst_buf.get(); copy_t = t_buf.get();
        } else {
            TTC_CUDA(cudaMemcpyAsync(src_buf.get(), src_in, m0 * 4, cudaMemcpyHostToDevice, s));
            TTC_CUDA(cudaMemcpyAsync(dst_buf.get(), dst_in, m0 * 4, cudaMemcpyHostToDevice, s));
            TTC_CUDA(cudaMemcpyAsync(t_buf.get(), t_in, m0 * 8, cudaMemcpyHostToDevice, s));
            in_src = src_buf.get(); in_dst = dst_buf.get(); in_t = t_buf.get();
        }
        src = src_buf.get(); dst = dst_buf.get(); t = t_buf.get();
    }
    DevBuf<IngestStats> ist(1, s);
    {
        IngestStats init{};
        init.tmin = LLONG_MAX;
        init.tmax = LLONG_MIN;
        TTC_CUDA(cudaMemcpyAsync(ist.get(), &init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    DevBuf<uint8_t> keep(m0 + 1, s);
    if (m0) {
        ingest_check_kernel<<<grid_for(m0), TPB, 0, s>>>(in_src, in_dst, in_t, m0, keep.get(), ist.get(), copy_src,
                                                        copy_dst, copy_t);
        TTC_LAUNCH_CHECK();
    }
    const IngestStats is = read_scalar(ist.get(), s);
    if (is.bad_id) fail(TTC_ERR_RANGE, "vertex id >= 2^31");
    if (is.bad_t) fail(TTC_ERR_RANGE, "timestamp outside [-2^62, 2^62]");
    st.m_self_loops = is.loops;
    const size_t m = m0 - (size_t)is.loops;
    st.m = m;
    const uint64_t n = m ? (uint64_t)is.max_id + 1 : 0;
    st.n = m0 ? (uint64_t)is.max_id + 1 : 0;
    // two keys of padding: the count kernels' bulk copies move whole 16-byte
    // words, so a list that ends on an odd key reads 8 bytes beyond it
    g->key.alloc(m + 2, s);
    g->fwd.alloc(m + 1, s);
    if (m == 0) {
        g->poff.alloc(1, s);
        TTC_CUDA(cudaMemsetAsync(g->poff.get(), 0, 4, s));
        TTC_CUDA(cudaMemsetAsync(g->fwd.get(), 0, 4, s));
        set_view(g, s);
        return;
    }

    g->tmin = is.tmin;
    g->span = is.tmax - is.tmin;
    const int span_bits = bits_for((uint64_t)g->span);
    const int ib = bits_for(m - 1);
    const bool direct = span_bits + ib + 1 <= 63;
    // kept edges in input order (index, time): with no self-loops and the
    // direct key they are the inputs themselves
    DevBuf<uint32_t> eidx;
    DevBuf<int64_t> tk;
    const uint32_t *eidx_p = nullptr;
    const int64_t *tk_p = t;
    if (is.loops || !direct) {
        eidx.alloc(m, s);
        tk.alloc(m, s);
        DevBuf<uint32_t> pos(m0 + 1, s);
        exclusive_scan_flags(keep.get(), pos.get(), m0, s);
        compact_kernel<<<grid_for(m0), TPB, 0, s>>>(keep.get(), pos.get(), m0, t, eidx.get(), tk.get());
        TTC_LAUNCH_CHECK();
        eidx_p = eidx.get();
        tk_p = tk.get();
    }
    keep.reset();

    prof_end(g, s);
    prof_begin(g, s, "load:keys_pair_sort");
    // ---- a2: per-edge key (t - t_min, tie rank, dir), grouped by pair and
    // key-sorted inside each pair by two stable sorts: time, then pair
    if (n * n > (uint64_t(1) << 63)) fail(TTC_ERR_RANGE, "vertex ids too large for the pair key");
    DevBuf<uint64_t> pkey(m, s);
    bool seg_sort_after = false;
    if (direct) {
        // ties broken by the kept-edge index itself (input order)
        g->shift = ib + 1;
        key_direct_kernel<<<grid_for(m), TPB, 0, s>>>(eidx_p, tk_p, m, g->tmin, g->shift, src, dst, n,
                                                      reinterpret_cast<uint64_t *>(g->key.get()), pkey.get());
        TTC_LAUNCH_CHECK();
        tk.reset(); eidx.reset();
        src_buf.reset(); dst_buf.reset(); t_buf.reset();
        // pairs are grouped first; each pair's keys are sorted below
        seg_sort_after = true;
    } else {
        // ties broken by the rank inside each equal-timestamp group
        DevBuf<uint64_t> tkey(m, s);
        time_key_kernel<<<grid_for(m), TPB, 0, s>>>(tk.get(), m, g->tmin, tkey.get(), eidx.get(), eidx.get());
        TTC_LAUNCH_CHECK();
        tk.reset();
        radix_sort_u64_u32(tkey.get(), eidx.get(), m, span_bits, s);
        DevBuf<uint8_t> head(m, s);
        DevBuf<uint32_t> gid(m + 1, s);
        head_flags_kernel<<<grid_for(m), TPB, 0, s>>>(tkey.get(), m, head.get());
        TTC_LAUNCH_CHECK();
        exclusive_scan_flags(head.get(), gid.get(), m, s);
        const uint32_t ngroups = read_scalar(gid.get() + m, s);
        DevBuf<uint32_t> gstart(ngroups ? ngroups : 1, s);
        group_start_kernel<<<grid_for(m), TPB, 0, s>>>(head.get(), gid.get(), m, gstart.get());
        TTC_LAUNCH_CHECK();
        DevBuf<unsigned int> maxr(1, s);
        TTC_CUDA(cudaMemsetAsync(maxr.get(), 0, 4, s));
        group_rank_max_kernel<<<grid_for(m), TPB, 0, s>>>(gid.get(), gstart.get(), m, maxr.get());
        TTC_LAUNCH_CHECK();
        const uint32_t max_rank = read_scalar(maxr.get(), s);
        g->shift = bits_for(max_rank) + 1;
        if (span_bits + g->shift > 63)
            fail(TTC_ERR_RANGE, "timestamp span needs %d bits plus %d tie bits; at most 63 fit the packed key",
                 span_bits, g->shift);
        pack_kernel<<<grid_for(m), TPB, 0, s>>>(tkey.get(), eidx.get(), gid.get(), gstart.get(), src, dst, m,
                                                g->shift, n, pkey.get(), reinterpret_cast<uint64_t *>(g->key.get()));
        TTC_LAUNCH_CHECK();
        src_buf.reset(); dst_buf.reset(); t_buf.reset();
    }
    st.key_bits = (uint32_t)(span_bits + g->shift);
    // group by pair; stable, so each pair's edges stay in key order
    radix_sort_bufs(pkey, g->key, m, 0, bits_for(n * n - 1), s);
    DevBuf<uint8_t> head(m, s);
    DevBuf<uint32_t> pid(m + 1, s);
    head_flags_kernel<<<grid_for(m), TPB, 0, s>>>(pkey.get(), m, head.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_flags(head.get(), pid.get(), m, s);
    const uint32_t ms = read_scalar(pid.get() + m, s);
    st.m_s = ms;
    g->poff.alloc((size_t)ms + 1, s);
    g->pair_vtx.alloc(ms, s);
    pair_rle_kernel<<<grid_for(m), TPB, 0, s>>>(pkey.get(), head.get(), pid.get(), m, n, g->poff.get(),
                                                g->pair_vtx.get());
    TTC_LAUNCH_CHECK();
    {
        const uint32_t mm32 = (uint32_t)m;
        TTC_CUDA(cudaMemcpyAsync(g->poff.get() + ms, &mm32, 4, cudaMemcpyHostToDevice, s));
        TTC_CUDA(cudaStreamSynchronize(s));
    }
    pid.reset(); head.reset(); pkey.reset();
    // ---- a5: each pair's list in key order and its dir-0 prefix.  Nothing
    // before the count reads them, so they run on a side stream that
    // overlaps the peel, orientation and enumeration, and join at the end.
    SideStream side(s);
    DevBuf<unsigned int> cls(3 * SEG_CLASSES, side.s);  // counts, bases, cursors
    DevBuf<uint32_t> lists(ms ? ms : 1, side.s);
    DevBuf<uint8_t> dflag(m, side.s);
    if (seg_sort_after) {
        unsigned int *cnt = cls.get(), *cbase = cnt + SEG_CLASSES, *cur = cbase + SEG_CLASSES;
        TTC_CUDA(cudaMemsetAsync(cnt, 0, SEG_CLASSES * 4, side.s));
        seg_classify_kernel<false><<<grid_for(ms), TPB, 0, side.s>>>(g->poff.get(), ms, cnt, nullptr);
        TTC_LAUNCH_CHECK();
        seg_bases_kernel<<<1, 1, 0, side.s>>>(cnt, cbase, cur);
        TTC_LAUNCH_CHECK();
        seg_classify_kernel<true><<<grid_for(ms), TPB, 0, side.s>>>(g->poff.get(), ms, cur, lists.get());
        TTC_LAUNCH_CHECK();
        seg_sort_tiny_kernel<<<grid_for(ms), TPB, 0, side.s>>>(g->key.get(), g->poff.get(), ms);
        TTC_LAUNCH_CHECK();
        seg_sort_classes(g->key.get(), g->poff.get(), lists.get(), cbase, cnt, side.s);
    }
    dir0_flags_kernel<<<grid_for(m), TPB, 0, side.s>>>(g->key.get(), m, dflag.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_flags(dflag.get(), g->fwd.get(), m, side.s);
    side.fork_done();

    prof_end(g, s);
    prof_begin(g, s, "load:degrees");
    // ---- static graph: undirected CSR, degrees
    DevBuf<unsigned int> deg(n, s), smax(1, s), lo_cnt(n, s), hi_cnt(n, s);
    DevBuf<uint32_t> lo_first(n, s);
    TTC_CUDA(cudaMemsetAsync(lo_cnt.get(), 0, n * 4, s));
    TTC_CUDA(cudaMemsetAsync(hi_cnt.get(), 0, n * 4, s));
    TTC_CUDA(cudaMemsetAsync(smax.get(), 0, 4, s));
    pair_sizes_kernel<<<grid_for(ms), TPB, 0, s>>>(g->poff.get(), ms, g->pair_vtx.get(), lo_first.get(), hi_cnt.get(),
                                                   smax.get());
    TTC_LAUNCH_CHECK();
    lo_runs_kernel<<<grid_for(ms), TPB, 0, s>>>(ms, g->pair_vtx.get(), lo_first.get(), lo_cnt.get());
    TTC_LAUNCH_CHECK();
    deg_sum_kernel<<<grid_for(n), TPB, 0, s>>>(n, lo_cnt.get(), hi_cnt.get(), deg.get());
    TTC_LAUNCH_CHECK();
    st.sigma_max = read_scalar(smax.get(), s);
    g->heavy_wide = st.sigma_max >= 65536;

    prof_end(g, s);
    prof_begin(g, s, "load:peel_adj");
    // ---- a3: ordering
    DevBuf<uint32_t> level(n, s);
    TTC_CUDA(cudaMemsetAsync(level.get(), 0xff, n * 4, s));
    if (opt.orientation == TTC_ORIENT_DEGENERACY) {
        if (2ull * ms >= (uint64_t(1) << 32)) fail(TTC_ERR_RANGE, "too many static edges for the peel");
        DevBuf<uint32_t> adj_off(n + 1, s), adj(2 * (size_t)ms, s);
        exclusive_scan_u32(deg.get(), adj_off.get(), n, s);
        TTC_CUDA(cudaMemsetAsync(hi_cnt.get(), 0, n * 4, s));  // now the cursors of the lower neighbours
        adj_fill_kernel<<<grid_for(ms), TPB, 0, s>>>(g->pair_vtx.get(), ms, adj_off.get(), lo_first.get(),
                                                     lo_cnt.get(), hi_cnt.get(), adj.get());
        TTC_LAUNCH_CHECK();
        lo_first.reset(); lo_cnt.reset(); hi_cnt.reset();
        prof_end(g, s);
        prof_begin(g, s, "load:peel_grid");
        DevBuf<int> pdeg(n, s);
        TTC_CUDA(cudaMemcpyAsync(pdeg.get(), deg.get(), n * 4, cudaMemcpyDeviceToDevice, s));
        DevBuf<uint32_t> remA(n, s), remB(n, s), frontA(n, s), frontB(n, s), foffA(n, s), foffB(n, s);
        DevBuf<PeelCtl> ctl(1, s);
        PeelCtl init{};
        for (auto &sl : init.slot) sl.min_deg = INT_MAX;
        TTC_CUDA(cudaMemcpyAsync(ctl.get(), &init, sizeof(init), cudaMemcpyHostToDevice, s));
        const uint32_t *a_off = adj_off.get(), *a_adj = adj.get();
        int *pd = pdeg.get();
        uint32_t *lv = level.get(), *rA = remA.get(), *rB = remB.get(), *fA = frontA.get(), *fB = frontB.get(),
                 *oA = foffA.get(), *oB = foffB.get();
        uint32_t n32 = (uint32_t)n;
        PeelCtl *pc = ctl.get();
        // stage 1: every SM, down to what the core cluster holds (one CTA when
        // cooperative launches are unavailable)
        {
            const int csize = core_cluster_size();
            if (csize <= 0) fail(TTC_ERR_CUDA, "no thread-block cluster of 8 or 16 CTAs fits this device");
            uint32_t stop = (uint32_t)csize * CORE_PER_MAX;
            void *args[] = {(void *)&a_off, (void *)&a_adj, (void *)&pd, (void *)&lv, (void *)&rA, (void *)&rB,
                            (void *)&fA, (void *)&fB, (void *)&oA, (void *)&oB, (void *)&n32, (void *)&stop,
                            (void *)&pc};
            const int grid_ctas = peel_grid_ctas();
            if (grid_ctas > 0)
                TTC_CUDA(cudaLaunchCooperativeKernel((const void *)peel_kernel, dim3(grid_ctas), dim3(PEEL_THREADS),
                                                     args, PEEL_SMEM, s));
            else
                TTC_CUDA(cudaLaunchKernel((const void *)peel_kernel, dim3(1), dim3(PEEL_THREADS), args, PEEL_SMEM, s));
            note_launch();
        }
        PeelCtl out = read_scalar(ctl.get(), s);
        if (out.error) fail(TTC_ERR_INTERNAL, "k-core peel did not finish");
        prof_end(g, s);
        prof_begin(g, s, "load:peel_core");
        if (out.handoff) {
            // stage 2, the core: the remaining vertices get local ids and their
            // induced adjacency; one cluster peels them down to PEEL_TAIL
            // vertices (peel_core_kernel), one CTA the rest (peel_tail_kernel)
            uint32_t R = out.rem_n;
            const uint32_t *rem = out.rem_in_b ? remB.get() : remA.get();
            uint32_t *lid = frontA.get(), *tail_list = frontB.get();  // free after the first stage
            for (int pass = 0; pass < 2 && R; pass++) {
                const bool one_cta = R <= PEEL_TAIL;
                DevBuf<uint32_t> cdeg(R, s), coff(R + 1, s);
                tail_ids_kernel<<<grid_for(R), TPB, 0, s>>>(rem, R, pdeg.get(), lid, cdeg.get());
                TTC_LAUNCH_CHECK();
                exclusive_scan_u32(cdeg.get(), coff.get(), R, s);
                const uint32_t ce = read_scalar(coff.get() + R, s);
                DevBuf<uint32_t> cadj(ce ? ce : 1, s);
                DevBuf<uint32_t> nchunk(R, s), chunk_pre(R + 1, s), cursor(R, s);
                tail_chunks_kernel<<<grid_for(R), TPB, 0, s>>>(rem, R, adj_off.get(), nchunk.get());
                TTC_LAUNCH_CHECK();
                exclusive_scan_u32(nchunk.get(), chunk_pre.get(), R, s);
                TTC_CUDA(cudaMemsetAsync(cursor.get(), 0, (size_t)R * 4, s));
                tail_adj_kernel<<<sm_count() * 8, 256, 0, s>>>(rem, R, chunk_pre.get(), adj_off.get(), adj.get(),
                                                               level.get(), lid, coff.get(), cursor.get(),
                                                               cadj.get());
                TTC_LAUNCH_CHECK();
                const int cluster = core_cluster_size();
                if (cluster <= 0) fail(TTC_ERR_CUDA, "no thread-block cluster of 8 or 16 CTAs fits this device");
                if (one_cta) {
                    peel_tail_kernel<<<1, CORE_TAIL_THREADS, tail_smem_bytes(R), s>>>(
                        rem, R, coff.get(), cadj.get(), level.get(), ctl.get());
                    TTC_LAUNCH_CHECK();
                    note_launch();
                    out = read_scalar(ctl.get(), s);
                    if (out.error) fail(TTC_ERR_INTERNAL, "k-core peel of the core did not finish");
                    break;
                }
                const uint32_t ncta = (uint32_t)cluster;
                uint32_t per = 1;  // vertices a cluster CTA owns: a power of two
                while (per * ncta < R) per <<= 1;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(ncta);
                cfg.blockDim = dim3(CORE_THREADS);
                cfg.dynamicSmemBytes = core_smem_bytes(per);
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = ncta;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                TTC_CUDA(cudaLaunchKernelEx(&cfg, peel_core_kernel, rem, R, per, (const uint32_t *)coff.get(),
                                            (const uint32_t *)cadj.get(), level.get(), pdeg.get(), PEEL_TAIL,
                                            tail_list, ctl.get()));
                note_launch();
                out = read_scalar(ctl.get(), s);
                if (out.error) fail(TTC_ERR_INTERNAL, "k-core peel of the core did not finish");
                if (!out.handoff) break;
                if (out.rem_n > PEEL_TAIL || out.core_alive != out.rem_n)
                    fail(TTC_ERR_INTERNAL, "k-core peel: inconsistent hand-off");
                R = out.rem_n;
                rem = tail_list;
            }
        }
        st.peel_rounds = out.rounds;
    }
    prof_end(g, s);
    prof_begin(g, s, "load:order_orient");
    // ranks: vertices sorted by ordering key, ties by id
    DevBuf<uint64_t> okey_v(n, s);
    DevBuf<uint32_t> id_of(n, s), rank_of(n, s);
    TTC_CUDA(cudaMemsetAsync(smax.get(), 0, 4, s));
    order_key_kernel<<<grid_for(n), TPB, 0, s>>>((uint32_t)n, opt.orientation, level.get(), deg.get(), opt.seed,
                                                 okey_v.get(), id_of.get(), smax.get());
    TTC_LAUNCH_CHECK();
    level.reset();
    radix_sort_bufs(okey_v, id_of, n, 0, bits_for(read_scalar(smax.get(), s)), s);
    okey_v.reset();
    rank_scatter_kernel<<<grid_for(n), TPB, 0, s>>>(id_of.get(), (uint32_t)n, rank_of.get());
    TTC_LAUNCH_CHECK();

    // ---- a4: orientation, out-CSR (lists sorted by rank) and in-CSR
    DevBuf<uint64_t> okey(ms, s);
    DevBuf<uint32_t> opair(ms, s);
    orient_kernel<<<grid_for(ms), TPB, 0, s>>>(g->pair_vtx.get(), ms, rank_of.get(), n, okey.get(), opair.get());
    TTC_LAUNCH_CHECK();
    rank_of.reset();
    radix_sort_bufs(okey, opair, ms, 0, bits_for(n * n - 1), s);
    DevBuf<uint32_t> out_off(n + 1, s), in_off(n + 1, s), osrc(ms, s), onbr(ms, s), in_e(ms, s);
    offsets_from_sorted_kernel<<<grid_for(n + 1), TPB, 0, s>>>(okey.get(), ms, n, (uint32_t)n, out_off.get());
    TTC_LAUNCH_CHECK();
    TTC_CUDA(cudaMemsetAsync(smax.get(), 0, 4, s));
    max_gap_kernel<<<grid_for(n), TPB, 0, s>>>(out_off.get(), n, smax.get());
    TTC_LAUNCH_CHECK();
    {
        DevBuf<uint64_t> tkey(ms, s);
        split_okey_kernel<<<grid_for(ms), TPB, 0, s>>>(okey.get(), ms, n, osrc.get(), onbr.get(), tkey.get(),
                                                       in_e.get());
        TTC_LAUNCH_CHECK();
        okey.reset();
        radix_sort_bufs(tkey, in_e, ms, 0, bits_for(n - 1), s);
        offsets_from_sorted_kernel<<<grid_for(n + 1), TPB, 0, s>>>(tkey.get(), ms, 1, (uint32_t)n, in_off.get());
        TTC_LAUNCH_CHECK();
    }
    st.kappa = read_scalar(smax.get(), s);
    deg.reset();

    prof_end(g, s);
    prof_begin(g, s, "load:enumerate");
    // ---- a6: triangles, written straight into the light and heavy bins.
    // With no threshold given, the tuned one for graphs of this shape (if
    // ttc_tune_light measured one on this GPU), else the default.
    if (!opt.light_max_pairs) g->light_max_pairs = tuned_light_max(st);
    st.light_max_pairs = g->light_max_pairs;
    const RecCtx rc{g->labeling, g->light_max_pairs};
    DevBuf<uint4> ocsr(ms, s);
    osig_kernel<<<grid_for(ms), TPB, 0, s>>>(opair.get(), osrc.get(), onbr.get(), id_of.get(), g->poff.get(), ms,
                                             ocsr.get());
    TTC_LAUNCH_CHECK();
    id_of.reset();
    opair.reset();
    const TriCsr tc{onbr.get(), ocsr.get(), out_off.get(), osrc.get(), in_off.get(), in_e.get()};
    // work items: (target v, 32 of its in-edges)
    DevBuf<uint32_t> nit(n, s), it_pre(n + 1, s);
    tri_items_count_kernel<<<grid_for(n), TPB, 0, s>>>(out_off.get(), in_off.get(), (uint32_t)n, nit.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_u32(nit.get(), it_pre.get(), n, s);
    const uint32_t nitems = read_scalar(it_pre.get() + n, s);
    DevBuf<uint2> items(nitems ? nitems : 1, s);
    tri_items_fill_kernel<<<grid_for(nitems), TPB, 0, s>>>(it_pre.get(), (uint32_t)n, nitems, items.get());
    TTC_LAUNCH_CHECK();
    nit.reset(); it_pre.reset();
    const uint32_t nv_cap = tri_nv_cap(st.kappa);
    DevBuf<unsigned long long> ws(7, s);
    TTC_CUDA(cudaMemsetAsync(ws.get(), 0, 56, s));
    uint64_t n_light = 0, tau = 0, n_rec_light = 0;  // n_rec_light: light records stored
    if (opt.flags & TTC_LOAD_STREAM) {
        // no light records: one scan pass for the statistics and the heavy
        // records; the oriented graph stays for the counts
        DevBuf<unsigned long long> hn(1, s);
        uint64_t cap = 1u << 20;  // heavy records are few; a second pass takes any excess
        for (int pass = 0; pass < 2; pass++) {
            TTC_CUDA(cudaMemsetAsync(hn.get(), 0, 8, s));
            TTC_CUDA(cudaMemsetAsync(ws.get(), 0, 56, s));
            g->tri.alloc(cap, s);
            EnumArgs ea{};
            ea.sums = ws.get();
            ea.heavy = g->tri.get();
            ea.heavy_n = hn.get();
            ea.heavy_cap = cap;
            launch_enum<ENUM_SCAN>(items.get(), nitems, tc, rc, ea, nv_cap, s);
            const uint64_t nh = read_scalar(hn.get(), s);
            if (nh <= cap) break;
            cap = nh;  // too many heavy triangles for the first guess: again, with room for all
        }
        uint64_t c[2];
        TTC_CUDA(cudaMemcpyAsync(c, ws.get() + 5, 16, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        n_light = c[0];
        tau = c[0] + c[1];
        if (tau >= (uint64_t(1) << 32)) fail(TTC_ERR_RANGE, "more than 2^32 static triangles");
        g->streamed = true;
        g->s_items = static_cast<DevBuf<uint2> &&>(items);
        g->s_nitems = nitems;
        g->s_ocsr = static_cast<DevBuf<uint4> &&>(ocsr);
        g->s_onbr = static_cast<DevBuf<uint32_t> &&>(onbr);
        g->s_osrc = static_cast<DevBuf<uint32_t> &&>(osrc);
        g->s_in_e = static_cast<DevBuf<uint32_t> &&>(in_e);
        g->s_out_off = static_cast<DevBuf<uint32_t> &&>(out_off);
        g->s_in_off = static_cast<DevBuf<uint32_t> &&>(in_off);
        // chunks of work items whose light records fit the collecting buffer
        DevBuf<uint64_t> room(nitems ? nitems : 1, s), rpre(nitems + 1, s);
        const TriCsr kept{g->s_onbr.get(), g->s_ocsr.get(), g->s_out_off.get(), g->s_osrc.get(), g->s_in_off.get(),
                          g->s_in_e.get()};
        if (nitems) {
            item_room_kernel<<<grid_for(nitems), TPB, 0, s>>>(g->s_items.get(), nitems, kept, room.get());
            TTC_LAUNCH_CHECK();
        }
        exclusive_scan_u64(room.get(), rpre.get(), nitems, s);
        std::vector<uint64_t> hp(nitems + 1);
        TTC_CUDA(cudaMemcpyAsync(hp.data(), rpre.get(), (nitems + 1) * 8, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        uint64_t chunk = stream_chunk_records();
        for (uint32_t it = 0; it < nitems; it++) chunk = std::max<uint64_t>(chunk, hp[it + 1] - hp[it]);
        g->s_chunk_cap = std::min<uint64_t>(chunk, std::max<uint64_t>(hp[nitems], 1));
        g->s_chunks.assign(1, 0u);
        for (uint32_t it = 0; it < nitems;) {
            // the longest run of items from `it` whose rooms fit the buffer
            const uint64_t lim = hp[it] + g->s_chunk_cap;
            const uint32_t end = (uint32_t)(std::upper_bound(hp.begin() + it + 1, hp.end(), lim) - hp.begin()) - 1;
            it = std::max(end, it + 1);
            g->s_chunks.push_back(it);
        }
    } else {
    // room per oriented edge, then one enumeration pass into it
    DevBuf<uint64_t> room(ms, s), resv(ms + 1, s);
    tri_room_kernel<<<grid_for(ms), TPB, 0, s>>>(osrc.get(), out_off.get(), ms, room.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_u64(room.get(), resv.get(), ms, s);
    room.reset();
    const uint64_t total_room = read_scalar(resv.get() + ms, s);
    DevBuf<uint4> sparse(total_room ? total_room : 1, s);
    DevBuf<uint32_t> cl(ms + 1, s), ch(ms + 1, s);
    DevBuf<uint64_t> loff(ms + 1, s), hoff(ms + 1, s), cl64(ms + 1, s), ch64(ms + 1, s);
    TTC_CUDA(cudaMemsetAsync(cl.get(), 0, (ms + 1) * 4, s));
    TTC_CUDA(cudaMemsetAsync(ch.get(), 0, (ms + 1) * 4, s));
    {
        EnumArgs ea{};
        ea.cnt_light = cl.get();
        ea.cnt_heavy = ch.get();
        ea.resv = resv.get();
        ea.sparse = sparse.get();
        ea.sums = ws.get();
        launch_enum<ENUM_WRITE>(items.get(), nitems, tc, rc, ea, nv_cap, s);
    }
    widen_kernel<<<grid_for(ms), TPB, 0, s>>>(cl.get(), ch.get(), ms, cl64.get(), ch64.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_u64(cl64.get(), loff.get(), ms, s);
    exclusive_scan_u64(ch64.get(), hoff.get(), ms, s);
    uint64_t nlh[2];
    TTC_CUDA(cudaMemcpyAsync(&nlh[0], loff.get() + ms, 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaMemcpyAsync(&nlh[1], hoff.get() + ms, 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    n_light = nlh[0];
    n_rec_light = n_light;
    tau = nlh[0] + nlh[1];
    if (tau >= (uint64_t(1) << 32)) fail(TTC_ERR_RANGE, "more than 2^32 static triangles");
    g->tri.alloc(tau, s);
    if (tau) {
        const unsigned grid_c = (unsigned)std::min<uint64_t>(ceil_div(ms, 32 * TRI_WARPS), (uint64_t)sm_count() * 8);
        tri_compact_kernel<<<grid_c, TRI_THREADS, 0, s>>>(resv.get(), cl.get(), ch.get(), loff.get(), hoff.get(),
                                                          n_light, ms, sparse.get(), g->tri.get());
        TTC_LAUNCH_CHECK();
    }
    }
    osrc.reset(); onbr.reset(); ocsr.reset(); out_off.reset(); in_off.reset(); in_e.reset();
    st.tau = tau;
    st.tau_light = n_light;
    st.tau_heavy = tau - n_light;

    prof_end(g, s);
    prof_begin(g, s, "load:classify");
    // ---- statistics and heavy-path offsets
    const uint64_t nh = st.tau_heavy;
    DevBuf<uint64_t> he(nh ? nh : 1, s);
    // the statistics were summed by the enumeration from the sigma words;
    // if one was capped they are taken again from the records
    unsigned long long hws[5];
    TTC_CUDA(cudaMemcpyAsync(hws, ws.get(), 40, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    if (hws[4] && !g->streamed) {
        TTC_CUDA(cudaMemsetAsync(ws.get(), 0, 32, s));
        record_stats_kernel<<<grid_for(tau), TPB, 0, s>>>(g->tri.get(), tau, n_light, g->poff.get(), he.get(),
                                                          ws.get());
        TTC_LAUNCH_CHECK();
        TTC_CUDA(cudaMemcpyAsync(hws, ws.get(), 32, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
    } else if (nh) {
        heavy_sizes_kernel<<<grid_for(nh), TPB, 0, s>>>(g->tri.get() + n_rec_light, nh, g->poff.get(), he.get());
        TTC_LAUNCH_CHECK();
    }
    st.work_bytes = hws[0];
    st.enum_elems = hws[1];
    st.work_bytes_heavy = hws[2];
    st.light_pairs = hws[3];
    // heavy records in three classes by size (one warp, one CTA, flat),
    // stably partitioned so each class is contiguous; the huge class last
    // the classes' caps and the one-CTA class's search form: given, else
    // tuned for graphs of this shape at this light threshold, else the
    // kernels' capacities and binary searches
    uint32_t wcap = warp_capacity(g->heavy_wide), ccap = fused_capacity(g->heavy_wide);
    uint32_t merge = opt.heavy_merge;
    {
        uint32_t tw = opt.heavy_warp_cap, tc = opt.heavy_cta_cap, aw = 0, ac = 0, am = 0;
        if ((!tw || !tc || !merge) && tuned_heavy_caps(st, g->light_max_pairs, &aw, &ac, &am)) {
            if (!tw) tw = aw;
            if (!tc) tc = ac;
            if (!merge) merge = am;
        }
        if (tw) wcap = std::min(wcap, tw);
        if (tc) ccap = std::min(ccap, tc);
        ccap = std::max(ccap, wcap);
    }
    st.heavy_warp_cap = wcap;
    st.heavy_cta_cap = ccap;
    st.heavy_merge = merge ? merge : TTC_HEAVY_BINARY;
    uint64_t n_huge = 0, n_hw = 0, n_hc = 0;
    if (nh) {
        DevBuf<uint8_t> f0(nh, s), f1(nh, s), f2(nh, s);
        DevBuf<uint32_t> p0(nh + 1, s), p1(nh + 1, s), p2(nh + 1, s);
        heavy_class_kernel<<<grid_for(nh), TPB, 0, s>>>(he.get(), nh, wcap, ccap, f0.get(), f1.get(), f2.get());
        TTC_LAUNCH_CHECK();
        exclusive_scan_flags(f0.get(), p0.get(), nh, s);
        exclusive_scan_flags(f1.get(), p1.get(), nh, s);
        exclusive_scan_flags(f2.get(), p2.get(), nh, s);
        uint32_t cnt[3];
        TTC_CUDA(cudaMemcpyAsync(&cnt[0], p0.get() + nh, 4, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaMemcpyAsync(&cnt[1], p1.get() + nh, 4, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaMemcpyAsync(&cnt[2], p2.get() + nh, 4, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        n_hw = cnt[0];
        n_hc = cnt[1];
        n_huge = cnt[2];
        DevBuf<uint4> part(nh, s);
        DevBuf<uint64_t> he2(nh, s);
        heavy_partition_kernel<<<grid_for(nh), TPB, 0, s>>>(g->tri.get() + n_rec_light, he.get(), f0.get(),
                                                            f1.get(), p0.get(), p1.get(), p2.get(), nh, n_hw, n_hc,
                                                            part.get(), he2.get());
        TTC_LAUNCH_CHECK();
        TTC_CUDA(cudaMemcpyAsync(g->tri.get() + n_rec_light, part.get(), nh * sizeof(uint4),
                                 cudaMemcpyDeviceToDevice, s));
        if (n_huge) {
            g->huge_eoff.alloc(n_huge + 1, s);
            exclusive_scan_u64(he2.get() + n_hw + n_hc, g->huge_eoff.get(), n_huge, s);
            g->huge_elems = read_scalar(g->huge_eoff.get() + n_huge, s);
        }
        TTC_CUDA(cudaStreamSynchronize(s));
    }
    st.tau_hwarp = n_hw;
    st.tau_hcta = n_hc;
    st.tau_huge = n_huge;
    // join the side stream; the pairs longer than the in-place sort's largest
    // class are sorted together (by key, then stably by pair), and the dir-0
    // prefix is taken again
    side.join();
    if (seg_sort_after) {
        unsigned int lp[2];  // count and list base of the pairs too long for the in-place sorts
        TTC_CUDA(cudaMemcpyAsync(&lp[0], cls.get() + SEG_CLASSES - 1, 4, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaMemcpyAsync(&lp[1], cls.get() + 2 * SEG_CLASSES - 1, 4, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        if (lp[0]) {
            const uint32_t nb = lp[0];
            DevBuf<uint32_t> start(nb, s);
            DevBuf<uint64_t> len(nb, s), pre((size_t)nb + 1, s);
            long_pair_list_kernel<<<grid_for(nb), TPB, 0, s>>>(lists.get() + lp[1], nb, g->poff.get(), start.get(),
                                                               len.get());
            TTC_LAUNCH_CHECK();
            exclusive_scan_u64(len.get(), pre.get(), nb, s);
            const uint64_t total = read_scalar(pre.get() + nb, s);
            DevBuf<uint64_t> gk(total, s), rk(total, s);
            DevBuf<uint32_t> gr(total, s);
            long_pair_gather_kernel<<<grid_for(total), TPB, 0, s>>>(g->key.get(), start.get(), pre.get(), nb, total,
                                                                    gk.get(), gr.get());
            TTC_LAUNCH_CHECK();
            radix_sort_u64_u32(gk.get(), gr.get(), total, (int)st.key_bits, s);
            long_pair_rank_kernel<<<grid_for(total), TPB, 0, s>>>(gr.get(), total, rk.get());
            TTC_LAUNCH_CHECK();
            radix_sort_u64_u64(rk.get(), gk.get(), total, bits_for(nb - 1), s);
            long_pair_scatter_kernel<<<grid_for(total), TPB, 0, s>>>(gk.get(), start.get(), pre.get(), nb, total,
                                                                     g->key.get());
            TTC_LAUNCH_CHECK();
            dir0_flags_kernel<<<grid_for(m), TPB, 0, s>>>(g->key.get(), m, dflag.get());
            TTC_LAUNCH_CHECK();
            exclusive_scan_flags(dflag.get(), g->fwd.get(), m, s);
        }
    }
    cls.reset(); lists.reset(); dflag.reset();
    set_view(g, s);
    prof_end(g, s);
    TTC_CUDA(cudaStreamSynchronize(s));
}

uint64_t stream_chunk_records() {
    const char *e = getenv("TTC_STREAM_CHUNK");
    const long long v = e ? atoll(e) : 0;
    return v > 0 ? (uint64_t)v : (uint64_t(1) << 24);
}

void stream_count_light(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s) {
    if (!g->streamed || !g->st.tau_light || !k) return;
    const TriCsr tc{g->s_onbr.get(), g->s_ocsr.get(), g->s_out_off.get(), g->s_osrc.get(), g->s_in_off.get(),
                    g->s_in_e.get()};
    const RecCtx rc{g->labeling, g->light_max_pairs};
    const uint64_t cap = g->s_chunk_cap;
    DevBuf<uint4> light(cap, s);
    DevBuf<unsigned long long> light_n(1, s);
    DevBuf<GraphView> view(1, s);
    DevBuf<uint64_t> pre(2, s);
    GraphView v = g->view_host;
    v.tri = light.get();
    TTC_CUDA(cudaMemcpyAsync(view.get(), &v, sizeof v, cudaMemcpyHostToDevice, s));
    for (size_t c = 0; c + 1 < g->s_chunks.size(); c++) {
        const uint32_t i0 = g->s_chunks[c], i1 = g->s_chunks[c + 1];
        TTC_CUDA(cudaMemsetAsync(light_n.get(), 0, 8, s));
        EnumArgs ea{};
        ea.light = light.get();
        ea.light_n = light_n.get();
        ea.light_cap = cap;
        prof_begin(g, s, "stream_collect");
        launch_enum<ENUM_COLLECT>(g->s_items.get() + i0, i1 - i0, tc, rc, ea, tri_nv_cap(g->st.kappa), s);
        prof_end(g, s);
        chunk_view_kernel<<<1, 1, 0, s>>>(light_n.get(), cap, view.get(), pre.get());
        TTC_LAUNCH_CHECK();
        count_light_records(g, view.get(), pre.get(), cap, dq, k, acc, s);
    }
}

}  // namespace ttc
