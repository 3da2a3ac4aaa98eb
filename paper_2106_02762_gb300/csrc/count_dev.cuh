// Device helpers of the per-query count (Alg. 1, counting step): the type
// table (Table 1 with Fig. 4), searches in key-sorted pair lists, counter
// updates with carry detection, and the light bin's per-pair count
// (Lemma 1 summed over A x B).  Shared by the count kernels and by the
// enumeration kernel when it counts light triangles as it finds them.
#pragma once

#include "graph.cuh"

namespace ttc {

namespace {

// Table 1 composed with Fig. 4, packed into one word per temporal ordering:
// bits 3 code .. 3 code + 2 of type_pack(pi) hold the type index (T_(value + 1))
// of psi(pi, rho(code)), where code = 4 dA + 2 dB + dC from the directions of
// the three pairs, direction 0 being u->v, u->w, v->w.  The lookup is then
// a shift of a compile-time word instead of a table load.
constexpr uint32_t type_pack(int pi) {
    // Table 1: psi(pi_k, rho_r); rows pi_1..pi_6, columns rho_1..rho_8
    const uint8_t psi[6][8] = {
        {6, 5, 4, 7, 2, 1, 3, 0},
        {4, 2, 6, 3, 5, 0, 7, 1},
        {2, 1, 0, 3, 6, 5, 7, 4},
        {0, 6, 2, 7, 1, 4, 3, 5},
        {5, 0, 1, 7, 4, 2, 3, 6},
        {1, 4, 5, 3, 0, 6, 7, 2},
    };
    // Fig. 4: rho_1 = (0,0,0), rho_2 = (0,1,1), rho_3 = (0,0,1), rho_4 = (0,1,0),
    // rho_5 = (1,0,0), rho_6 = (1,1,1), rho_7 = (1,0,1), rho_8 = (1,1,0) as (dA, dB, dC)
    const uint8_t rho_of_code[8] = {0, 2, 3, 1, 4, 6, 7, 5};
    uint32_t v = 0;
    for (int code = 0; code < 8; code++) v |= uint32_t(psi[pi][rho_of_code[code]]) << (3 * code);
    return v;
}

// Temporal orderings (Fig. 3), 0-based: pi_1 = A,B,C  pi_2 = B,A,C  pi_3 = A,C,B
// pi_4 = B,C,A  pi_5 = C,A,B  pi_6 = C,B,A  (first, second, third pair).
enum { PI1 = 0, PI2 = 1, PI3 = 2, PI4 = 3, PI5 = 4, PI6 = 5 };
constexpr uint32_t TP1 = type_pack(PI1), TP2 = type_pack(PI2), TP3 = type_pack(PI3), TP4 = type_pack(PI4),
                   TP5 = type_pack(PI5), TP6 = type_pack(PI6);
// every row of Table 1 is a permutation of the eight types
constexpr bool packs_types_once(uint32_t pack) {
    uint32_t seen = 0;
    for (int code = 0; code < 8; code++) seen |= 1u << ((pack >> (3 * code)) & 7u);
    return seen == 0xffu;
}
static_assert(packs_types_once(TP1) && packs_types_once(TP2) && packs_types_once(TP3) && packs_types_once(TP4) &&
                  packs_types_once(TP5) && packs_types_once(TP6),
              "Table 1 rows are permutations");

__device__ __forceinline__ uint32_t pack_of(int pi) {
    return pi == PI1 ? TP1 : pi == PI2 ? TP2 : pi == PI3 ? TP3 : pi == PI4 ? TP4 : pi == PI5 ? TP5 : TP6;
}
__device__ __forceinline__ int type_in(uint32_t pack, uint32_t code) { return (int)((pack >> (3 * code)) & 7u); }
__device__ __forceinline__ int type_of(int pi, uint32_t dA, uint32_t dB, uint32_t dC) {
    return type_in(pack_of(pi), (dA << 2) | (dB << 1) | dC);
}

struct Query {
    int64_t d13, d12, d23;
};

// ---------------------------------------------------------------- index checks
// A build with -DTTC_DEBUG_BOUNDS=1 (the stand-in for a device memory
// checker) checks, before a list is used, every pair id read from a
// triangle record against the number of pairs and every list's range
// against the key array, and every bulk copy's range against the array and
// its padding.  A failed check sets g_bounds_bad, the triangle is not
// counted (no access is made), and the count call returns
// TTC_ERR_INTERNAL.  Searches stay inside a checked range by construction.
#ifndef TTC_DEBUG_BOUNDS
#define TTC_DEBUG_BOUNDS 0
#endif
static __device__ unsigned int g_bounds_bad;

// true when [.., hi) lies below lim (always, unless checking)
__device__ __forceinline__ bool in_range(uint64_t hi, uint64_t lim) {
    if (!TTC_DEBUG_BOUNDS || hi <= lim) return true;
    atomicOr(&g_bounds_bad, 1u);
    return false;
}

__device__ __forceinline__ Query load_query(const int64_t *dq, uint32_t q) {
    return Query{dq[3 * q], dq[3 * q + 1], dq[3 * q + 2]};
}

// ---------------------------------------------------------------- lists
// A pair's key-sorted edge list in device memory: key[b .. b + n), with the
// direction split read from the global dir-0 prefix `fwd`.
// number of keys < bound in the sorted p[0 .. n)
__device__ __forceinline__ uint32_t search_below(const int64_t *__restrict__ p, uint32_t n, int64_t bound) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (__ldg(p + lo + half) < bound) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

struct GList {
    const int64_t *__restrict__ key;
    const uint32_t *__restrict__ fwd;
    uint32_t b, n, flip;  // flip: effective direction = stored ^ 1
    // number of keys < bound (bound >= 0)
    __device__ __forceinline__ uint32_t below(int64_t bound) const { return search_below(key + b, n, bound); }
    // effective direction-0 edges among the first pos
    __device__ __forceinline__ uint32_t d0(uint32_t pos) const {
        const uint32_t s0 = __ldg(fwd + b + pos) - __ldg(fwd + b);
        return flip ? pos - s0 : s0;
    }
};

// A list staged in shared memory: keys and an effective dir-0 prefix
// (d0(i) = d0p[i] - base = direction-0 edges among the first i).
struct SList {
    const int64_t *key;
    const uint32_t *d0p;
    uint32_t n, base;
    __device__ __forceinline__ uint32_t below(int64_t bound) const {
        uint32_t lo = 0, len = n;
        while (len > 0) {
            const uint32_t half = len >> 1;
            if (key[lo + half] < bound) {
                lo += half + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        return lo;
    }
    __device__ __forceinline__ uint32_t d0(uint32_t pos) const { return d0p[pos] - base; }
};

// Packed-key format ((t - t_min) << shift | tie << 1 | dir) for time bounds.
struct KeyFmt {
    int shift;
    int64_t span;
    // Def. 1's t1 < t2 < t3 read literally: "after" is a later timestamp,
    // not a later key (t, input index)
    bool strict;
};
// #{e in L : key(e) < key(x)} for an edge x not in L
template <typename L>
__device__ __forceinline__ uint32_t cnt_key(const L &l, int64_t kx) {
    return l.below(kx & ~int64_t(1));
}
// #{e in L : t(e) - t_min <= x}
template <typename L>
__device__ __forceinline__ uint32_t cnt_le(const L &l, const KeyFmt &f, int64_t x) {
    if (x < 0) return 0;
    if (x >= f.span) return l.n;
    return l.below((x + 1) << f.shift);
}
// #{e in L : t(e) - t_min < x}
template <typename L>
__device__ __forceinline__ uint32_t cnt_lt(const L &l, const KeyFmt &f, int64_t x) {
    return cnt_le(l, f, x - 1);
}

// Search bounds, as keys: #{e : key(e) < bound} gives cnt_key, cnt_le and
// cnt_lt.  Every key is >= 0 and below INT64_MAX, so bound 0 counts nothing
// and INT64_MAX counts the whole list.
__device__ __forceinline__ int64_t key_bound(int64_t kx) { return kx & ~int64_t(1); }
__device__ __forceinline__ int64_t le_bound(const KeyFmt &f, int64_t x) {
    return x < 0 ? 0 : x >= f.span ? INT64_MAX : (x + 1) << f.shift;
}
__device__ __forceinline__ int64_t lt_bound(const KeyFmt &f, int64_t x) { return le_bound(f, x - 1); }

// res[i] = #{keys < bound[i]} in a sorted list of n keys (at(i) reads key
// i), for N bounds at once.  The halving steps depend only on n, so the N
// searches advance in lockstep and their loads are in flight together.
template <int N, typename AT>
__device__ __forceinline__ void search_n(AT &&at, uint32_t n, const int64_t (&bound)[N], uint32_t (&res)[N]) {
#pragma unroll
    for (int i = 0; i < N; i++) res[i] = 0;
    uint32_t len = n;  // each answer lies in [res[i], res[i] + len]
    while (len > 1) {
        const uint32_t half = len >> 1;
        int64_t v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = at(res[i] + half - 1);
#pragma unroll
        for (int i = 0; i < N; i++) res[i] += v[i] < bound[i] ? half : 0u;
        len -= half;
    }
    if (len == 1) {
        int64_t v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = at(res[i]);
#pragma unroll
        for (int i = 0; i < N; i++) res[i] += v[i] < bound[i] ? 1u : 0u;
    }
}
// search_n for the bounds whose bit is set in `mask` (the others are not
// searched: their lanes issue no loads and res stays 0).
template <int N, typename AT>
__device__ __forceinline__ void search_n_masked(AT &&at, uint32_t n, const int64_t (&bound)[N], uint32_t mask,
                                                uint32_t (&res)[N]) {
#pragma unroll
    for (int i = 0; i < N; i++) res[i] = 0;
    uint32_t len = n;
    while (len > 1) {
        const uint32_t half = len >> 1;
        int64_t v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = (mask >> i & 1u) ? at(res[i] + half - 1) : INT64_MAX;
#pragma unroll
        for (int i = 0; i < N; i++) res[i] += v[i] < bound[i] ? half : 0u;
        len -= half;
    }
    if (len == 1) {
        int64_t v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = (mask >> i & 1u) ? at(res[i]) : INT64_MAX;
#pragma unroll
        for (int i = 0; i < N; i++) res[i] += v[i] < bound[i] ? 1u : 0u;
    }
}
template <int N>
__device__ __forceinline__ void search_n(const GList &l, const int64_t (&bound)[N], uint32_t (&res)[N]) {
    const int64_t *p = l.key + l.b;
    search_n<N>([&](uint32_t i) { return __ldg(p + i); }, l.n, bound, res);
}
template <int N>
__device__ __forceinline__ void search_n(const SList &l, const int64_t (&bound)[N], uint32_t (&res)[N]) {
    search_n<N>([&](uint32_t i) { return l.key[i]; }, l.n, bound, res);
}

__device__ __forceinline__ GList glist(const GraphView &gv, uint32_t p, uint32_t flip) {
    if (!in_range((uint64_t)p + 1, gv.ms)) return GList{gv.key, gv.fwd, 0u, 0u, flip};
    const uint32_t b = __ldg(gv.poff + p);
    const uint32_t n = __ldg(gv.poff + p + 1) - b;
    if (!in_range((uint64_t)b + n, gv.m)) return GList{gv.key, gv.fwd, 0u, 0u, flip};
    return GList{gv.key, gv.fwd, b, n, flip};
}

// ---------------------------------------------------------------- bulk copies
// Global -> shared copies by the bulk-copy engine (cp.async.bulk), tracked
// by a transaction-count mbarrier in shared memory.  Both addresses must be
// 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory
// before later bulk copies into it (after a barrier, for the whole CTA's).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One arrival that also expects `bytes` of bulk-copy transactions.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Waits for the phase with parity `parity` to complete, for at most `limit`
// polls; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bit of the count calls' device flag word set when a bounded wait gave up
// (bit 0 is the overflow bit).
constexpr unsigned long long FLAG_TIMEOUT = 2ull;

// ---------------------------------------------------------------- accumulation
__device__ __forceinline__ void add_checked(unsigned long long &acc, unsigned long long x, unsigned &ovf) {
    const unsigned long long r = acc + x;
    ovf |= r < acc;
    acc = r;
}

// Adds this warp's per-thread counters s_acc[type][tid] into out[0..8) with
// one atomic per type, zeroes them, and raises *flag on any carry.  Every
// lane of the warp must call it.
__device__ __forceinline__ void warp_flush(unsigned long long (*s_acc)[256], unsigned long long *out,
                                           unsigned long long *flag, unsigned &ovf) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 8; t++) {
        unsigned long long v = s_acc[t][threadIdx.x];
        s_acc[t][threadIdx.x] = 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
            add_checked(v, y, ovf);
        }
        if (lane == 0 && v) {
            const unsigned long long old = atomicAdd(out + t, v);
            ovf |= old + v < old;
        }
    }
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(flag, 1ull);
    ovf = 0;
}

// The same for 32-bit per-thread counters s_c[type][tid] whose carries went
// to this warp's 64-bit words s_w[type] (see add_u32_carry).
__device__ __forceinline__ void warp_flush32(uint32_t (*s_c)[256], unsigned long long *s_w,
                                             unsigned long long *out, unsigned long long *flag, unsigned &ovf) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 8; t++) {
        unsigned long long v = s_c[t][threadIdx.x];
        s_c[t][threadIdx.x] = 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);  // 32 terms < 2^32: no carry
        __syncwarp();
        if (lane == 0) {
            add_checked(v, s_w[t], ovf);
            s_w[t] = 0;
            if (v) {
                const unsigned long long old = atomicAdd(out + t, v);
                ovf |= old + v < old;
            }
        }
    }
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(flag, 1ull);
    ovf = 0;
}

// A 32-bit per-thread counter: a carry out of it adds 2^32 to the 64-bit
// accumulator `wide` (a shared atomic, rare).
__device__ __forceinline__ void add_u32_carry(uint32_t &cell, uint32_t n, unsigned long long *wide, unsigned &ovf) {
    const uint32_t old = cell;
    cell = old + n;
    if (cell < old) {
        const unsigned long long o = atomicAdd(wide, 1ull << 32);
        ovf |= o + (1ull << 32) < o;
    }
}

// A 32-bit per-thread counter whose carries go to a 64-bit word of the
// warp (shared by its lanes, hence the atomic).
__device__ __forceinline__ void add_wide32(uint32_t &cell, unsigned long long n, unsigned long long *wide,
                                           unsigned &ovf) {
    const unsigned long long hi = n >> 32;
    const uint32_t lo = (uint32_t)n, old = cell;
    cell = old + lo;
    const unsigned long long carry = hi + (cell < old ? 1ull : 0ull);
    if (carry) {
        const unsigned long long o = atomicAdd(wide, carry << 32);
        ovf |= (carry >> 32) != 0 || o + (carry << 32) < o;
    }
}

// Block accumulators (several queries): shared atomics with carry checks.
__device__ __forceinline__ void shared_add(unsigned long long *p, unsigned long long n, unsigned &ovf) {
    const unsigned long long old = atomicAdd(p, n);
    ovf |= old + n < old;
}

__device__ __forceinline__ void block_flush(const unsigned long long *s, uint32_t cnt, unsigned long long *out,
                                            unsigned long long *flag, unsigned ovf) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        if (s[i]) {
            const unsigned long long old = atomicAdd(out + i, s[i]);
            ovf |= old + s[i] < old;
        }
    }
    if (ovf) atomicOr(flag, 1ull);
}

// Graph of a global work index, from an exclusive prefix over graphs.
__device__ __forceinline__ uint32_t graph_of(const uint64_t *__restrict__ pre, uint32_t G, uint64_t i) {
    uint32_t lo = 0, hi = G;  // last g with pre[g] <= i
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// C's key-sorted list seen from one pair (x, y) of enumerated edges, x the
// earlier: px, py = #{c : key(c) < key(x)}, #{c : key(c) < key(y)}, and the
// raw dir-0 prefix fwd[b + pos] at pos = 0, px, py, n, the four positions
// that bound every case of Lemma 1 once its window is unbounded.
struct CView {
    const int64_t *__restrict__ key;
    const uint32_t *__restrict__ fwd;
    uint32_t b, n, flip;
    uint32_t px, py, f0, fx, fy, fn;
    int64_t kfirst, klast;  // C's first and last keys (when loaded; else 0 and INT64_MAX)
    // a short list read whole: bit j of mask0 is set when C's key j has
    // stored direction 0, and the raw prefix is counted from it (from 0, so
    // every raw value of the list is on the same footing)
    bool small;
    uint32_t mask0;
    __device__ __forceinline__ uint32_t below(int64_t bound) const { return search_below(key + b, n, bound); }
    __device__ __forceinline__ uint32_t raw(uint32_t pos) const {
        if (small) return __popc(mask0 & ((1u << pos) - 1u));
        return pos == px ? fx : pos == py ? fy : pos == n ? fn : pos == 0 ? f0 : __ldg(fwd + b + pos);
    }
    // effective direction-0 edges among C's positions [lo, hi)
    __device__ __forceinline__ uint32_t d0_range(uint32_t lo, uint32_t hi) const {
        const uint32_t s = raw(hi) - raw(lo);
        return flip ? (hi - lo) - s : s;
    }
};

// Adds the counts of one pair (x, y) of enumerated edges (x earlier, times
// rx <= ry) for all three positions of C's edge.  xa: x is on A (else on B).
// code = 4 dA + 2 dB (Fig. 4 with dC = 0).
template <bool LOCKSTEP, typename Acc>
__device__ __forceinline__ void light_pair(const CView &C, const KeyFmt &f, const Query &q, bool xa, int64_t rx,
                                           int64_t ry, uint32_t code, Acc &&acc) {
    if (!f.strict && q.d12 >= f.span && q.d23 >= f.span) {
        // every window covers the graph's whole time span (then so does d13
        // >= d12): C's edges after y, between x and y, and before x make the
        // three cases whole
        auto add_raw = [&](uint32_t pack, uint32_t len, uint32_t s) {  // s: raw dir-0 count of the range
            const uint32_t n0 = C.flip ? len - s : s;
            acc(type_in(pack, code), n0);
            acc(type_in(pack, code | 1u), len - n0);
        };
        if (C.n > C.py) add_raw(xa ? TP1 : TP2, C.n - C.py, C.fn - C.fy);
        if (C.py > C.px) add_raw(xa ? TP3 : TP4, C.py - C.px, C.fy - C.fx);
        if (C.px > 0) add_raw(xa ? TP5 : TP6, C.px, C.fx - C.f0);
        return;
    }
    const int64_t gap = ry - rx;
    // every case needs t_y - t_x <= d13 (d12, d23 <= d13 once normalised);
    // in the strict reading x and y at one time have no order
    if (gap > q.d13 || (f.strict && gap == 0)) return;
    if constexpr (!LOCKSTEP) {
        // one search per window end, each when its case can count (fewer
        // registers than the lockstep form, for kernels that keep state for
        // several queries)
        const uint32_t ay = f.strict ? cnt_le(C, f, ry) : C.py, by = f.strict ? cnt_lt(C, f, ry) : C.py;
        const uint32_t ax = f.strict ? cnt_le(C, f, rx) : C.px, bx = f.strict ? cnt_lt(C, f, rx) : C.px;
        auto add = [&](uint32_t pack, uint32_t lo, uint32_t hi) {
            const uint32_t n0 = C.d0_range(lo, hi);
            acc(type_in(pack, code), n0);
            acc(type_in(pack, code | 1u), (hi - lo) - n0);
        };
        if (gap <= q.d12) {  // C third
            const uint32_t hi = cnt_le(C, f, min(ry + q.d23, rx + q.d13));
            if (hi > ay) add(xa ? TP1 : TP2, ay, hi);
        }
        {  // C second (gap <= d13 here)
            const uint32_t lo = max(ax, cnt_lt(C, f, ry - q.d23));
            const uint32_t hi = min(by, cnt_le(C, f, rx + q.d12));
            if (hi > lo) add(xa ? TP3 : TP4, lo, hi);
        }
        if (gap <= q.d23) {  // C first
            const uint32_t lo = cnt_lt(C, f, max(rx - q.d12, ry - q.d13));
            if (bx > lo) add(xa ? TP5 : TP6, lo, bx);
        }
        return;
    }
    // the window ends of the three cases, found by one lockstep search (a
    // case whose gap condition fails gets bound 0, which needs no load):
    //   C third  [after y, le(min(ry + d23, rx + d13)))
    //   C second [max(after x, lt(ry - d23)), min(before y, le(rx + d12)))
    //   C first  [lt(max(rx - d12, ry - d13)), before x)
    // In the strict reading "after" and "before" are time bounds too.
    constexpr int NB = 8;
    const int64_t b[NB] = {gap <= q.d12 ? le_bound(f, min(ry + q.d23, rx + q.d13)) : 0,
                           gap <= q.d13 ? lt_bound(f, ry - q.d23) : 0,
                           gap <= q.d13 ? le_bound(f, rx + q.d12) : 0,
                           gap <= q.d23 ? lt_bound(f, max(rx - q.d12, ry - q.d13)) : 0,
                           f.strict ? le_bound(f, ry) : 0, f.strict ? lt_bound(f, ry) : 0,
                           f.strict ? le_bound(f, rx) : 0, f.strict ? lt_bound(f, rx) : 0};
    // a bound at or below C's first key counts nothing and one above its
    // last key counts all of C; only the others are searched
    uint32_t p[NB], mask = 0;
#pragma unroll
    for (int i = 0; i < NB; i++) {
        p[i] = b[i] <= C.kfirst ? 0u : b[i] > C.klast ? C.n : 0u;
        if (b[i] > C.kfirst && b[i] <= C.klast && (f.strict || i < 4)) mask |= 1u << i;
    }
    if (mask) {
        uint32_t sp[NB];
        if (f.strict) {
            search_n_masked<8>([&](uint32_t i) { return __ldg(C.key + C.b + i); }, C.n, b, mask, sp);
        } else {
            const int64_t b4[4] = {b[0], b[1], b[2], b[3]};
            uint32_t s4[4];
            search_n_masked<4>([&](uint32_t i) { return __ldg(C.key + C.b + i); }, C.n, b4, mask, s4);
#pragma unroll
            for (int i = 0; i < 4; i++) sp[i] = s4[i];
        }
#pragma unroll
        for (int i = 0; i < NB; i++)
            if (mask >> i & 1u) p[i] = sp[i];
    }
    // C's edges after y start at ay, those before y end at by; likewise x
    const uint32_t ay = f.strict ? p[4] : C.py, by = f.strict ? p[5] : C.py;
    const uint32_t ax = f.strict ? p[6] : C.px, bx = f.strict ? p[7] : C.px;
    auto add = [&](uint32_t pack, uint32_t lo, uint32_t hi) {
        const uint32_t n0 = C.d0_range(lo, hi);
        acc(type_in(pack, code), n0);
        acc(type_in(pack, code | 1u), (hi - lo) - n0);
    };
    if (gap <= q.d12 && p[0] > ay) add(xa ? TP1 : TP2, ay, p[0]);  // C third
    if (gap <= q.d13) {                                            // C second
        const uint32_t lo = max(ax, p[1]), hi = min(by, p[2]);
        if (hi > lo) add(xa ? TP3 : TP4, lo, hi);
    }
    if (gap <= q.d23 && bx > p[3]) add(xa ? TP5 : TP6, p[3], bx);  // C first
}

// One (a, b) pair of a light triangle (Lemma 1 over A x B): a = A's edge ai
// (A's list starts at key[ab]), b = B's edge bi (at key[bb]), C = key[cb ..
// cb + cn), fl the record's flip flags.  have_ends: f0 = fwd[cb] and
// fn = fwd[cb + cn] are given, else loaded here.  A pair whose time gap
// exceeds gmax (the largest d13 of the queries at hand) is skipped;
// otherwise each(C, a_first, rx, ry, code) runs light_pair for each query.
// gfin: the largest d13 of the queries whose windows do not cover the whole
// time span (-1 if none).
template <uint32_t SHORT_C, typename EACH>
__device__ __forceinline__ void light_count_pair(const GraphView &gv, const KeyFmt &f, uint32_t ab, uint32_t bb,
                                                 uint32_t cb, uint32_t cn, uint32_t fl, bool have_ends, uint32_t f0,
                                                 uint32_t fn, uint32_t ai, uint32_t bi, int64_t gmax, int64_t gfin,
                                                 EACH &&each) {
    const int64_t ka = __ldg(gv.key + ab + ai), kb = __ldg(gv.key + bb + bi);
    // a list of at most SHORT_C keys is read whole (one memory round trip)
    // and its positions and direction counts are taken in registers
    // When the largest d13 at hand covers the whole time span no pair is
    // skipped, and the list is loaded with the pair's keys; otherwise after
    // the gap test, so that skipped pairs load nothing.
    const bool shortc = SHORT_C > 0 && cn <= SHORT_C;
    const bool early = gmax >= f.span;
    int64_t sk[SHORT_C > 0 ? SHORT_C : 1];
    if (shortc && early) {
#pragma unroll
        for (uint32_t j = 0; j < SHORT_C; j++) sk[j] = j < cn ? __ldg(gv.key + cb + j) : INT64_MAX;
    }
    const int64_t ra = ka >> f.shift, rb = kb >> f.shift;
    const bool a_first = ka < kb;
    const int64_t gap = a_first ? rb - ra : ra - rb;
    if (gap > gmax) return;
    if (shortc && !early) {
#pragma unroll
        for (uint32_t j = 0; j < SHORT_C; j++) sk[j] = j < cn ? __ldg(gv.key + cb + j) : INT64_MAX;
    }
    const uint32_t dA = (uint32_t)(ka & 1) ^ (fl & TriRec::FLIP_A);
    const uint32_t dB = (uint32_t)(kb & 1) ^ ((fl & TriRec::FLIP_B) ? 1u : 0u);
    const uint32_t code = (dA << 2) | (dB << 1);
    CView C;
    C.key = gv.key;
    C.fwd = gv.fwd;
    C.b = cb;
    C.n = cn;
    C.flip = (fl & TriRec::FLIP_C) ? 1u : 0u;
    if (shortc) {
        const int64_t ba = key_bound(ka), bbd = key_bound(kb);
        uint32_t pa = 0, pb = 0, mask = 0;
        int64_t last = sk[0];
#pragma unroll
        for (uint32_t j = 0; j < SHORT_C; j++) {
            pa += sk[j] < ba;
            pb += sk[j] < bbd;
            mask |= ((uint32_t)~sk[j] & 1u) << j;  // padding (INT64_MAX) is odd: no bit
            if (j < cn) last = sk[j];
        }
        C.small = true;
        C.mask0 = mask;
        C.px = a_first ? pa : pb;
        C.py = a_first ? pb : pa;
        C.f0 = 0;
        C.fx = __popc(mask & ((1u << C.px) - 1u));
        C.fy = __popc(mask & ((1u << C.py) - 1u));
        C.fn = __popc(mask);
        C.kfirst = sk[0];
        C.klast = last;
    } else {
        // C's first and last keys settle most window ends without a search;
        // only a query with finite windows and d13 >= gap can need them
        // (gfin: the largest d13 of such queries, -1 if none).  Loaded
        // before the key searches, they arrive while those run.
        const bool ends = gap <= gfin;
        C.kfirst = ends ? __ldg(gv.key + cb) : 0;
        C.klast = ends ? __ldg(gv.key + cb + cn - 1) : INT64_MAX;
        const int64_t *ck = gv.key + cb;
        const int64_t bab[2] = {key_bound(ka), key_bound(kb)};
        uint32_t pab[2];
        search_n<2>([&](uint32_t i) { return __ldg(ck + i); }, cn, bab, pab);
        C.small = false;
        C.mask0 = 0;
        C.px = a_first ? pab[0] : pab[1];
        C.py = a_first ? pab[1] : pab[0];
        C.f0 = have_ends ? f0 : __ldg(gv.fwd + cb);
        C.fn = have_ends ? fn : __ldg(gv.fwd + cb + cn);
        C.fx = __ldg(gv.fwd + cb + C.px);
        C.fy = __ldg(gv.fwd + cb + C.py);
    }
    each(C, a_first, a_first ? ra : rb, a_first ? rb : ra, code);
}

}  // namespace

}  // namespace ttc
