// Per-query counting (Alg. 1, counting step): for every static triangle
// <u, v, w> and every temporal ordering pi and orientation rho, the number of
// (d13, d12, d23)-temporal triangles, added to the type psi(pi, rho)
// (Table 1).  Only the edge lists of the pairs A = {u, v} and B = {u, w} are
// enumerated; the list of C = {v, w} is only searched (Sec. 5).
//
// Three bins, chosen per triangle at load time:
//
// light  (sigma_A * sigma_B small): Lemma 1 summed directly over the pairs
//        (a, b) in A x B.  With x the earlier and y the later of a, b (key
//        order), C's edge c can be
//          third  (x, y, c): t_y - t_x <= d12, key(c) > key(y),
//                            t_c <= min(t_y + d23, t_x + d13)      (Lemma 1)
//          second (x, c, y): t_y - t_x <= d13, key(x) < key(c) < key(y),
//                            t_c <= t_x + d12, t_c >= t_y - d23
//          first  (c, x, y): t_y - t_x <= d23, key(c) < key(x),
//                            t_c >= max(t_x - d12, t_y - d13)
//        and each case is a contiguous index range of C's key-sorted list.
//        A warp flattens the pairs of 32 triangles across its lanes.
//
// heavy  the prefix-sum form of Algs. 2-4, re-derived with key order for
//        ties.  Each enumerated edge e of A or B first gets, per direction of
//        C,
//          h(e) = #{c: t_c <= t_e + d13}          (CEC_{+d13} terms, Alg. 2)
//          L(e) = #{c: key(c) < key(e)}           (CEC_{-inf} terms, Alg. 3)
//          R(e) = #{c: t_c <  t_e - d23}          (CEC_{-d23} terms, Alg. 3)
//          M(e) = #{c: t_c <  t_e - d13}          (CEC_{-d13} terms, Alg. 4)
//        (phase 1); their prefix sums over each list and own direction are
//        then read at binary-searched range ends while every edge of the
//        other list is enumerated (phase 2).  One CTA takes one triangle:
//        both lists and all prefix sums stay in shared memory.
//
// huge   heavy triangles whose two lists do not fit one CTA: the same
//        phases, flat over every enumerated edge of every huge triangle (so
//        one triangle is spread over many CTAs), prefix sums in device
//        scratch.
//
// Deltas arrive normalised (d12, d23 <= d13 <= d12 + d23); all counts are
// unsigned 64-bit sums with carry detection.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "graph.cuh"
#include "count_dev.cuh"

namespace ttc {

namespace {

// ---------------------------------------------------------------- light bin
constexpr int LIGHT_THREADS = 256;
constexpr uint32_t LIGHT_QT = 2;  // queries per group kept in per-thread accumulators
constexpr int LIGHT_WARPS = LIGHT_THREADS / 32;
// Records per lane in one work item of a batched (MODE 1) launch: a warp
// takes 32 * LIGHT_BATCH_R triangles, so the last, partly filled round of
// their flattened pairs is a smaller share of the rounds.  (Measured on the
// power-law workload: one record per lane is faster for single queries, two
// for batches.)
constexpr int LIGHT_BATCH_R = 2;
// Records per lane in one work item of a single-query (MODE 0) launch on
// one graph (measured on the power-law workload: two beat one and four).
constexpr int LIGHT_SINGLE_R = 2;
// Length classes of C's list (at most 4, 16, 64 edges, longer) by which a
// work item orders its triangles.
constexpr uint32_t LIGHT_CLASSES = 4;

template <int R>
struct WarpTris {
    uint32_t excl[LIGHT_WARPS][32 * R + 1];  // exclusive prefix of pair counts
    uint4 lst[LIGHT_WARPS][32 * R];          // A.b, B.b, C.b, C.n
    uint32_t aux[LIGHT_WARPS][32 * R];       // B.n | flip flags << 29 (B.n < 2^20 in the light bin)
    uint8_t orig[LIGHT_WARPS][32 * R];       // MODE 2: the record's place in the item
    Query q[LIGHT_WARPS][LIGHT_QT];          // MODE 1: the item's query group
};

// Warp-cooperative light kernel over a table of graphs.  Each warp takes
// 32 R consecutive triangle records (record base + r * 32 + lane in slot
// r * 32 + lane), flattens their A x B pairs into one index space and gives
// every lane one pair per round.
//   MODE 0: one query per graph (dq[3 g]); out[8 g + type].
//   MODE 1: nq queries on graph 0; out[8 q + type].
//   MODE 2: one query on graph 0 for the triangles idx[0 .. nidx);
//           out[8 i + type] per triangle.
// chunk_pre[g] = first 32-record chunk of graph g (exclusive prefix, G + 1);
// R > 1 needs G == 1.  Every light triangle has sigma_A * sigma_B below the
// light threshold (at most 2^20), so a work item has fewer than 2^32 pairs
// and a pair's index within its triangle is below 2^20.
template <int MODE, int R, bool ST>
__global__ void __launch_bounds__(LIGHT_THREADS, 4)
    light_kernel(const GraphView *__restrict__ gvs, const uint64_t *__restrict__ chunk_pre, uint32_t G,
                 const int64_t *dq, uint32_t nq, unsigned long long *out, unsigned long long *flag,
                 const uint64_t *idx, uint64_t nidx, uint32_t qpw = 1) {
    __shared__ WarpTris<R> wt;
    // MODE 0: per-thread 32-bit counters; a carry out of one adds 2^32 to
    // its warp's 64-bit word (warps of one block may be on different graphs)
    __shared__ uint32_t s_acc[MODE == 0 ? 8 : 1][MODE == 0 ? 256 : 1];
    __shared__ unsigned long long s_wide[MODE == 0 ? LIGHT_WARPS : 1][8];
    // MODE 1: [nq * 8] block accumulators, then, when every item's query
    // group has at most LIGHT_QT queries, per-thread 32-bit accumulators
    // [LIGHT_QT * 8][LIGHT_THREADS] (no shared atomics per pair; a carry out
    // of one adds 2^32 to the block accumulator, and 32-bit cells keep the
    // block's shared memory small enough for four blocks per SM)
    extern __shared__ unsigned long long s_bacc[];
    const bool tslots = MODE == 1 && qpw <= LIGHT_QT;
    uint32_t *s_t = reinterpret_cast<uint32_t *>(s_bacc + 8 * (size_t)nq);
    uint32_t slot_q0 = 0;  // first query of the group the thread's slots hold
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
        if ((threadIdx.x & 31) < 8) s_wide[threadIdx.x >> 5][threadIdx.x & 31] = 0;
    }
    // MODE 1 without thread slots: the queries in descending d13 order (ties
    // by index), so that a pair stops at the first query whose d13 is below
    // its time gap (every later one would skip it too; a query whose windows
    // cover the time span has d13 >= span >= any gap, so it comes first)
    Query *s_qs = reinterpret_cast<Query *>(s_t);
    uint32_t *s_qi = reinterpret_cast<uint32_t *>(s_qs + nq);
    if constexpr (MODE == 1) {
        for (uint32_t i = threadIdx.x; i < nq * 8; i += blockDim.x) s_bacc[i] = 0;
        if (tslots) {
            for (uint32_t i = 0; i < LIGHT_QT * 8; i++) s_t[i * LIGHT_THREADS + threadIdx.x] = 0;
        } else {
            for (uint32_t i = threadIdx.x; i < nq; i += blockDim.x) {
                const int64_t di = dq[3 * i];
                uint32_t r = 0;
                for (uint32_t j = 0; j < nq; j++) {
                    const int64_t dj = dq[3 * j];
                    r += (dj > di || (dj == di && j < i)) ? 1u : 0u;
                }
                s_qs[r] = load_query(dq, i);
                s_qi[r] = i;
            }
        }
        __syncthreads();
    }

    unsigned ovf = 0;
    uint32_t cur_g = 0xffffffffu;
    // adds the thread's slots into the block accumulators of queries
    // slot_q0 .. slot_q0 + qpw - 1 (warp sums first) and clears them
    auto flush_slots = [&]() {
        for (uint32_t ql = 0; ql < qpw && slot_q0 + ql < nq; ql++) {
#pragma unroll
            for (int t = 0; t < 8; t++) {
                uint32_t &cell = s_t[(ql * 8 + t) * LIGHT_THREADS + threadIdx.x];
                unsigned long long v = cell;
                cell = 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
                    add_checked(v, y, ovf);
                }
                if (lane == 0 && v) shared_add(&s_bacc[(slot_q0 + ql) * 8 + t], v, ovf);
            }
        }
    };
    constexpr uint32_t PER = 32 * R;  // records per work item
    const uint64_t nchunks = MODE == 2 ? (nidx + PER - 1) / PER
                             : R == 1 ? __ldg(chunk_pre + G)
                                      : (__ldg(chunk_pre + 1) + R - 1) / R;
    const uint64_t gw = (uint64_t)blockIdx.x * LIGHT_WARPS + w, nw = (uint64_t)gridDim.x * LIGHT_WARPS;
    // MODE 1: work items are (chunk, group of qpw queries), so small graphs
    // still spread a large batch over many warps
    const uint32_t ngroups = MODE == 1 ? (nq + qpw - 1) / qpw : 1u;
    for (uint64_t item = gw; item < nchunks * ngroups; item += nw) {
        const uint64_t c = item / ngroups;
        const uint32_t q_beg = MODE == 1 ? (uint32_t)(item % ngroups) * qpw : 0u;
        const uint32_t q_end = MODE == 1 ? min(nq, q_beg + qpw) : 1u;
        if (MODE == 1 && tslots && q_beg != slot_q0) {  // warp-uniform
            flush_slots();
            slot_q0 = q_beg;
        }
        const uint32_t g = MODE == 0 && R == 1 ? graph_of(chunk_pre, G, c) : 0u;
        if constexpr (MODE == 0) {
            if (g != cur_g) {
                if (cur_g != 0xffffffffu) warp_flush32(s_acc, s_wide[w], out + 8 * cur_g, flag, ovf);
                cur_g = g;
            }
        }
        const GraphView &gv = gvs[g];
        const KeyFmt f{gv.shift, gv.span, ST};
        // the group's queries (MODE 1: in the warp's shared slots when the
        // thread's accumulators hold them)
        Query Q0{0, 0, 0};
        int64_t gmax = 0;  // every case needs t_y - t_x <= d13
        if constexpr (MODE == 1) {
            if (tslots && lane < q_end - q_beg) wt.q[w][lane] = load_query(dq, q_beg + lane);
            for (uint32_t q = q_beg; q < q_end; q++) gmax = max(gmax, dq[3 * q]);
        } else {
            Q0 = load_query(dq, MODE == 0 ? g : 0u);
            gmax = Q0.d13;
        }
        // the largest d13 of the item's queries with a window shorter than the
        // time span (-1 if none): pairs within it load C's end keys
        // (the batched kernel searches window ends one by one and loads no end
        // keys: it keeps state for several queries and has no registers to spare)
        int64_t gfin = -1;
        if constexpr (MODE != 1) {
            if (ST || Q0.d12 < gv.span || Q0.d23 < gv.span) gfin = Q0.d13;
        }
        const uint64_t base = (MODE == 0 && R == 1 ? c - __ldg(chunk_pre + g) : c) * PER;
        const uint64_t lim = MODE == 2 ? nidx : gv.n_light;
        uint32_t np[R], cls[R];
        uint4 lst[R];
        uint32_t aux[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const uint32_t slot = r * 32 + lane;
            const uint64_t ti = base + slot;
            np[r] = 0;
            cls[r] = 0;
            lst[r] = make_uint4(0, 0, 0, 0);
            aux[r] = 0;
            if (ti < lim) {
                const uint4 rec = __ldg(gv.tri + (MODE == 2 ? idx[ti] : ti));
                const uint32_t pm = max(rec.x, max(rec.y, rec.z));
                const bool ok = in_range((uint64_t)pm + 1, gv.ms);
                const uint32_t ab = ok ? __ldg(gv.poff + rec.x) : 0u, an = ok ? __ldg(gv.poff + rec.x + 1) - ab : 0u;
                const uint32_t bb = ok ? __ldg(gv.poff + rec.y) : 0u, bn = ok ? __ldg(gv.poff + rec.y + 1) - bb : 0u;
                const uint32_t cb = ok ? __ldg(gv.poff + rec.z) : 0u, cn = ok ? __ldg(gv.poff + rec.z + 1) - cb : 0u;
                const bool lists_ok = ok && in_range((uint64_t)ab + an, gv.m) && in_range((uint64_t)bb + bn, gv.m) &&
                                      in_range((uint64_t)cb + cn, gv.m) && cn > 0;
                np[r] = lists_ok ? an * bn : 0u;
                cls[r] = cn <= 4 ? 0u : cn <= 16 ? 1u : cn <= 64 ? 2u : 3u;
                lst[r] = make_uint4(ab, bb, cb, cn);
                aux[r] = bn | (rec.w << 29);
            }
        }
        // the item's triangles in order of the length class of C (counting
        // sort by ballots): a round of pairs then covers C lists of similar
        // length, so its lanes' searches take about the same number of steps
        {
            const uint32_t below = (1u << lane) - 1u;
            uint32_t done = 0, pos[R];
#pragma unroll
            for (uint32_t k = 0; k < LIGHT_CLASSES; k++) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const uint32_t m = __ballot_sync(0xffffffffu, cls[r] == k);
                    if (cls[r] == k) pos[r] = done + __popc(m & below);
                    done += __popc(m);
                }
            }
#pragma unroll
            for (int r = 0; r < R; r++) {
                wt.lst[w][pos[r]] = lst[r];
                wt.aux[w][pos[r]] = aux[r];
                wt.excl[w][pos[r]] = np[r];
                if constexpr (MODE == 2) wt.orig[w][pos[r]] = (uint8_t)(r * 32 + lane);
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; r++) np[r] = wt.excl[w][r * 32 + lane];
            __syncwarp();
        }
        uint32_t total = 0;
#pragma unroll
        for (int r = 0; r < R; r++) {
            uint32_t x = np[r];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            wt.excl[w][r * 32 + lane] = total + x - np[r];
            total += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) wt.excl[w][PER] = total;
        __syncwarp();
        for (uint32_t rbase = 0; rbase < total; rbase += 32) {
            const uint32_t j = rbase + lane;
            if (j >= total) continue;
            uint32_t o = 0;  // last slot with excl <= j (skips empty slots before it)
#pragma unroll
            for (uint32_t step = PER / 2; step; step >>= 1)
                if (wt.excl[w][o + step] <= j) o += step;
            const uint4 L = wt.lst[w][o];
            const uint32_t X = wt.aux[w][o], bn = X & ((1u << 29) - 1), fl = X >> 29;
            const uint32_t loc = j - wt.excl[w][o];
            // loc < 2^20: (loc + 1/2) / bn is at least 1 / (2 bn) from an
            // integer, and the float product is within 2^-3 / bn of it
            const uint32_t ai = __float2uint_rz(((float)loc + 0.5f) * __frcp_rn((float)bn)), bi = loc - ai * bn;
            light_count_pair<MODE == 1 ? 4u : 2u>(gv, f, L.x, L.y, L.z, L.w, fl, false, 0u, 0u, ai, bi, gmax, gfin,
                             [&](const CView &C, bool a_first, int64_t rx, int64_t ry, uint32_t code) {
                if (MODE != 1 || tslots) {
#pragma unroll 1
                    for (uint32_t ql = 0; ql < (MODE == 1 ? LIGHT_QT : 1u); ql++) {
                        if (MODE == 1 && q_beg + ql >= q_end) break;
                        auto accq = [&](int type, uint32_t n) {
                            if constexpr (MODE == 0) add_u32_carry(s_acc[type][threadIdx.x], n, &s_wide[w][type], ovf);
                            else if constexpr (MODE == 1)
                                add_u32_carry(s_t[(ql * 8 + type) * LIGHT_THREADS + threadIdx.x], n,
                                              &s_bacc[(q_beg + ql) * 8 + type], ovf);
                            else atomicAdd(out + 8 * (base + wt.orig[w][o]) + type, (unsigned long long)n);
                        };
                        light_pair<MODE != 1>(C, f, MODE == 1 ? wt.q[w][ql] : Q0, a_first, rx, ry, code, accq);
                    }
                } else {
                    const int64_t gap = ry - rx;
                    for (uint32_t r = 0; r < nq && s_qs[r].d13 >= gap; r++) {
                        const uint32_t q = s_qi[r];
                        if (q - q_beg >= q_end - q_beg) continue;  // outside [q_beg, q_end)
                        auto accq = [&](int type, uint32_t n) { shared_add(&s_bacc[q * 8 + type], n, ovf); };
                        light_pair<false>(C, f, s_qs[r], a_first, rx, ry, code, accq);
                    }
                }
            });
        }
        __syncwarp();
    }
    if constexpr (MODE == 0) {
        if (cur_g != 0xffffffffu) warp_flush32(s_acc, s_wide[w], out + 8 * cur_g, flag, ovf);
    }
    if constexpr (MODE == 1) {
        if (tslots) flush_slots();
        block_flush(s_bacc, nq * 8, out, flag, ovf);
    }
}

// ---------------------------------------------------------------- heavy: per-edge math
// Searches of the two phases, binary or two-pointer.  Along one enumerated
// list in key order every bound the phases look up in C or in the other
// list is a non-decreasing function of the edge's time or key (t_e plus a
// constant window end, or the key itself), so each answer #{keys < bound}
// only moves forward from one edge to the next.  The two-pointer form gives
// a thread a contiguous run of edges of one list: the first edge's bounds
// are binary-searched, every later edge's are found by stepping forward from
// the previous answers.  The answers are the same either way, so the prefix
// sums of Algs. 2-4 read at them are too.
template <int N>
struct Cursor {
    uint32_t pos[N];
    bool valid;  // pos holds the answers for the previous edge of the same list
};

__device__ __forceinline__ int64_t list_key(const SList &l, uint32_t i) { return l.key[i]; }
__device__ __forceinline__ int64_t list_key(const GList &l, uint32_t i) { return __ldg(l.key + l.b + i); }

// res[i] = #{keys < bd[i]} in l; with a cursor, stepped forward from its
// answers when it holds some (the bounds must not be below the previous
// ones), and left holding these answers.
template <int N, typename L>
__device__ __forceinline__ void find_n(const L &l, const int64_t (&bd)[N], uint32_t (&res)[N], Cursor<N> *cur) {
    if (cur && cur->valid) {
#pragma unroll
        for (int i = 0; i < N; i++) {
            uint32_t p = cur->pos[i];
            while (p < l.n && list_key(l, p) < bd[i]) p++;
            res[i] = p;
        }
    } else {
        search_n<N>(l, bd, res);
    }
    if (cur) {
#pragma unroll
        for (int i = 0; i < N; i++) cur->pos[i] = res[i];
        cur->valid = true;
    }
}

// Phase 1 for an enumerated edge e (key ke): the values h, L, R, M against C,
// each split by C's direction: out[2 s + dC].
template <typename CL>
__device__ __forceinline__ void phase1_values(const CL &C, const KeyFmt &f, const Query &q, int64_t ke,
                                              uint32_t out[8], Cursor<4> *cur = nullptr) {
    const int64_t re = ke >> f.shift;
    // L(e): C's edges before e, by key or (strict) by time
    const int64_t bd[4] = {le_bound(f, re + q.d13), f.strict ? lt_bound(f, re) : key_bound(ke),
                           lt_bound(f, re - q.d23), lt_bound(f, re - q.d13)};
    uint32_t ps[4];
    find_n<4>(C, bd, ps, cur);
    const uint32_t ph = ps[0], pl = ps[1], pr = ps[2], pm = ps[3];
    const uint32_t h0 = C.d0(ph), l0 = C.d0(pl), r0 = C.d0(pr), m0 = C.d0(pm);
    out[0] = h0; out[1] = ph - h0;
    out[2] = l0; out[3] = pl - l0;
    out[4] = r0; out[5] = pr - r0;
    out[6] = m0; out[7] = pm - m0;
}

// Phase 1 without L(e), which does not depend on the query: the batched
// kernels take it (and its prefix sums) from the batch's first query and
// search only h, R and M for the others (slots 2 and 3 of out untouched).
template <typename CL>
__device__ __forceinline__ void phase1_values_hrm(const CL &C, const KeyFmt &f, const Query &q, int64_t ke,
                                                  uint32_t out[8], Cursor<3> *cur = nullptr) {
    const int64_t re = ke >> f.shift;
    const int64_t bd[3] = {le_bound(f, re + q.d13), lt_bound(f, re - q.d23), lt_bound(f, re - q.d13)};
    uint32_t ps[3];
    find_n<3>(C, bd, ps, cur);
    const uint32_t ph = ps[0], pr = ps[1], pm = ps[2];
    const uint32_t h0 = C.d0(ph), r0 = C.d0(pr), m0 = C.d0(pm);
    out[0] = h0; out[1] = ph - h0;
    out[4] = r0; out[5] = pr - r0;
    out[6] = m0; out[7] = pm - m0;
}

// Phase 2 for an enumerated edge e with O the other enumerated list.
// pref(dO, s, c) = prefix over O's own-direction-dO edges, first c of them,
// of phase-1 slot s.  add(dO, dC, pi if e is on A, pi if e is on B, n).
// cc, co: cursors of the two-pointer form for the searches in C and in O.
template <typename OL, typename CL, typename PF, typename ADD>
__device__ __forceinline__ void phase2_edge(const OL &O, const CL &C, const KeyFmt &f, const Query &q, int64_t ke,
                                            PF &&pref, ADD &&add, Cursor<4> *cc = nullptr, Cursor<8> *co = nullptr) {
    const int64_t re = ke >> f.shift;
    // searches in C (split by C's direction).  C's edges not after e (Ka)
    // and before e (Kb): the same key position, or (strict) those with
    // t <= t_e and t < t_e
    const int64_t bc[4] = {f.strict ? le_bound(f, re) : key_bound(ke), le_bound(f, re + q.d23),
                           le_bound(f, re + q.d12), lt_bound(f, re - q.d12)};
    uint32_t pc[4];
    find_n<4>(C, bc, pc, cc);
    const uint32_t posCa = pc[0], pH = pc[1], pG = pc[2], pLo = pc[3];
    const uint32_t posCb = f.strict ? C.below(lt_bound(f, re)) : posCa;
    const uint32_t Ka0 = C.d0(posCa), H0 = C.d0(pH), G0 = C.d0(pG), Lo0 = C.d0(pLo);
    const uint32_t Kb0 = f.strict ? C.d0(posCb) : Ka0;
    const uint32_t Ka[2] = {Ka0, posCa - Ka0}, Kb[2] = {Kb0, posCb - Kb0}, Hd[2] = {H0, pH - H0},
                   Gd[2] = {G0, pG - G0}, Lod[2] = {Lo0, pLo - Lo0};
    // searches in O (merged positions)
    const int64_t bo[8] = {f.strict ? le_bound(f, re) : key_bound(ke),
                           lt_bound(f, re - q.d12),
                           le_bound(f, re + q.d23 - q.d13),
                           le_bound(f, re + min(q.d12, q.d23)),
                           le_bound(f, re + max(q.d12, q.d23)),
                           le_bound(f, re + q.d13),
                           le_bound(f, re + q.d13 - q.d12),
                           le_bound(f, re + q.d23)};
    uint32_t po[8];
    find_n<8>(O, bo, po, co);
    // O's edges before e end at posOb, those after e start at posOa: one
    // key position, or (strict) t < t_e and t <= t_e
    const uint32_t posOa = po[0], posOb = f.strict ? O.below(lt_bound(f, re)) : posOa;
    const uint32_t o_lo = min(po[1], posOb);
    const uint32_t o_mid = min(max(po[2], o_lo), posOb);
    const uint32_t r1 = max(po[3], posOa);
    const uint32_t r2 = max(po[4], r1);
    const uint32_t r3 = max(po[5], r2);
    const uint32_t sp = max(po[6], posOa);
    const uint32_t en = max(po[7], sp);
    const uint32_t pos[9] = {o_lo, o_mid, posOb, r1, r2, r3, sp, en, posOa};
    uint32_t d0s[9];
#pragma unroll
    for (int i = 0; i < 8; i++) d0s[i] = O.d0(pos[i]);
    d0s[8] = f.strict ? O.d0(posOa) : d0s[2];
#pragma unroll
    for (uint32_t dO = 0; dO < 2; dO++) {
        // own-direction-dO ranks of the merged positions in O
        uint32_t c[9];
#pragma unroll
        for (int i = 0; i < 9; i++) c[i] = dO ? pos[i] - d0s[i] : d0s[i];
        const uint32_t c_lo = c[0], c_mid = c[1], c_pb = c[2], c_r1 = c[3], c_r2 = c[4], c_r3 = c[5], c_sp = c[6],
                       c_en = c[7], c_pa = c[8];
#pragma unroll
        for (uint32_t dC = 0; dC < 2; dC++) {
            // (1) e second, O's edge first, C third: Alg. 2 (pi_2 if e is on A, pi_1 if on B)
            {
                const unsigned long long hsum = pref(dO, 0 + dC, c_mid) - pref(dO, 0 + dC, c_lo);
                const unsigned long long n = hsum + (unsigned long long)Hd[dC] * (c_pb - c_mid) -
                                             (unsigned long long)Ka[dC] * (c_pb - c_lo);
                add(dO, dC, PI2, PI1, n);
            }
            // (2) e first, C second, O's edge third: Alg. 3 (pi_3 / pi_4)
            {
                unsigned long long n = pref(dO, 2 + dC, c_r1) - pref(dO, 2 + dC, c_pa) -
                                       (unsigned long long)Ka[dC] * (c_r1 - c_pa);
                if (q.d12 <= q.d23) {
                    n += (unsigned long long)(Gd[dC] - Ka[dC]) * (c_r2 - c_r1);
                } else {
                    n += (pref(dO, 2 + dC, c_r2) - pref(dO, 2 + dC, c_r1)) -
                         (pref(dO, 4 + dC, c_r2) - pref(dO, 4 + dC, c_r1));
                }
                n += (unsigned long long)Gd[dC] * (c_r3 - c_r2) - (pref(dO, 4 + dC, c_r3) - pref(dO, 4 + dC, c_r2));
                add(dO, dC, PI3, PI4, n);
            }
            // (3) C first, e second, O's edge third: Alg. 4 (pi_5 / pi_6)
            {
                unsigned long long n = (unsigned long long)(Kb[dC] - Lod[dC]) * (c_sp - c_pa);
                n += (unsigned long long)Kb[dC] * (c_en - c_sp) - (pref(dO, 6 + dC, c_en) - pref(dO, 6 + dC, c_sp));
                add(dO, dC, PI5, PI6, n);
            }
        }
    }
}

// ---------------------------------------------------------------- heavy: fused CTA kernel
constexpr int HEAVY_THREADS = 256;
constexpr int HEAVY_WARPS = HEAVY_THREADS / 32;
constexpr uint32_t MAX_BATCH_SMEM_Q = 256;

template <typename P>
struct FusedCap {
    static constexpr uint32_t CAP = sizeof(P) == 4 ? 2048 : 1024;  // edges of A plus B
    static constexpr uint32_t ES = CAP + 4;                         // prefix entries per slot
    static constexpr uint32_t CC = 1024;                            // C lists up to this long are staged too
    static constexpr size_t KEYS = ((size_t)CAP + 4) * 8;            // A and B, each padded to 16-byte words
    static constexpr size_t D0 = ((size_t)CAP + 8) * 4;
    static constexpr size_t PRE = 8 * (size_t)ES * sizeof(P);
    static constexpr size_t CKEYS = ((size_t)CC + 2) * 8;            // C, padded to 16-byte words
    static constexpr size_t CD0 = ((size_t)CC + 8) * 4;
    // MODE 0 tail: 32-bit per-thread counters and one 64-bit carry word per
    // (warp, type); MODE 1: the queries' block accumulators
    static constexpr size_t TAIL0 = 8 * 256 * 4 + HEAVY_WARPS * 8 * 8;
    static constexpr size_t bytes(int mode, uint32_t nq) {
        return KEYS + D0 + PRE + CKEYS + CD0 + (mode == 1 ? (size_t)nq * 64 : mode == 0 ? TAIL0 : 0);
    }
};

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *tmp) {
    // tmp: HEAVY_WARPS + 1 words of shared memory; tmp[HEAVY_WARPS] = total
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < HEAVY_WARPS; i++) {
            const uint32_t t = tmp[i];
            tmp[i] = run;
            run += t;
        }
        tmp[HEAVY_WARPS] = run;
    }
    __syncthreads();
    return tmp[w] + x - v;
}

// One CTA per heavy triangle of the CTA class, over a table of graphs.  MODE
// as light_kernel; heavy_pre[g] = first CTA-class record of graph g in the
// global index space (G + 1 entries).  merge: take the two-pointer form for
// the triangles whose C is staged and holds at most as many edges as A and B
// together (the bounds then move little from one edge to the next).
template <typename P, int MODE, bool ST>
__global__ void __launch_bounds__(HEAVY_THREADS)
    heavy_fused_kernel(const GraphView *__restrict__ gvs, const uint64_t *__restrict__ heavy_pre, uint32_t G,
                       const int64_t *dq, uint32_t nq, unsigned long long *out, unsigned long long *flag,
                       const uint64_t *idx, uint64_t nidx, uint32_t merge) {
    using Cap = FusedCap<P>;
    constexpr uint32_t CAP = Cap::CAP, ES = Cap::ES;
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t *s_key = reinterpret_cast<int64_t *>(smem);
    uint32_t *s_d0 = reinterpret_cast<uint32_t *>(smem + Cap::KEYS);
    P *s_pre = reinterpret_cast<P *>(smem + Cap::KEYS + Cap::D0);
    int64_t *s_ck = reinterpret_cast<int64_t *>(smem + Cap::KEYS + Cap::D0 + Cap::PRE);
    uint32_t *s_cd0 = reinterpret_cast<uint32_t *>(smem + Cap::KEYS + Cap::D0 + Cap::PRE + Cap::CKEYS);
    unsigned long long *s_tail =
        reinterpret_cast<unsigned long long *>(smem + Cap::KEYS + Cap::D0 + Cap::PRE + Cap::CKEYS + Cap::CD0);
    auto s_acc = reinterpret_cast<uint32_t (*)[256]>(s_tail);                        // MODE 0
    unsigned long long *s_wide = s_tail + 8 * 256 / 2 + (threadIdx.x >> 5) * 8;  // MODE 0: this warp's carries
    __shared__ uint32_t s_tmp[HEAVY_WARPS + 1];
    __shared__ __align__(8) uint64_t s_bar;
    uint32_t bar_phase = 0;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    if constexpr (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
        if ((threadIdx.x & 31) < 8) s_wide[threadIdx.x & 31] = 0;
    }
    if constexpr (MODE == 1) {
        for (uint32_t i = threadIdx.x; i < nq * 8; i += blockDim.x) s_tail[i] = 0;
    }
    __syncthreads();
    unsigned ovf = 0;
    uint32_t cur_g = 0xffffffffu;
    const uint64_t nitems = MODE == 2 ? nidx : __ldg(heavy_pre + G);
    for (uint64_t h = blockIdx.x; h < nitems; h += gridDim.x) {
        const uint32_t g = MODE == 0 ? graph_of(heavy_pre, G, h) : 0u;
        if constexpr (MODE == 0) {
            if (g != cur_g) {
                if (cur_g != 0xffffffffu) warp_flush32(s_acc, s_wide, out + 8 * cur_g, flag, ovf);
                cur_g = g;
            }
        }
        const GraphView &gv = gvs[g];
        const KeyFmt f{gv.shift, gv.span, ST};
        const uint64_t hl = MODE == 2 ? idx[h] : (MODE == 0 ? h - __ldg(heavy_pre + g) : h);
        const uint4 r = __ldg(gv.tri + gv.n_light + gv.n_hwarp + hl);
        const GList A = glist(gv, r.x, r.w & TriRec::FLIP_A);
        const GList B = glist(gv, r.y, (r.w & TriRec::FLIP_B) ? 1u : 0u);
        const GList C = glist(gv, r.z, (r.w & TriRec::FLIP_C) ? 1u : 0u);
        const uint32_t na = A.n, nb = B.n, ne = na + nb;
        // block-uniform skips: lists beyond this kernel's capacity (never, by
        // the load-time partition), or a graph served by the other width
        if (ne > CAP || (sizeof(P) == 8) != (gv.wide != 0)) continue;
        // a C list up to CC edges is staged too, so both phases search it in
        // shared memory; a longer one is searched where it lies
        const bool c_staged = C.n <= Cap::CC;  // block-uniform
        // stage A, B (and C when staged) by bulk copies of whole 16-byte
        // words: A's keys at s_key[ao ..), B's at s_key[aw + bo ..), C's at
        // s_ck[co ..) (ao, bo, co: the lists' odd starts); the key array has
        // padding for the last word
        const uint32_t ao = A.b & 1u, bo = B.b & 1u, co = C.b & 1u;
        const uint32_t aw = (ao + na + 1u) & ~1u, bw = (bo + nb + 1u) & ~1u;
        const uint32_t cw = c_staged ? (co + C.n + 1u) & ~1u : 0u;
        // the copies end at most one key past a list, inside the padding
        if (!(in_range((uint64_t)A.b - ao + aw, gv.m + 2) && in_range((uint64_t)B.b - bo + bw, gv.m + 2) &&
              in_range((uint64_t)C.b - co + cw, gv.m + 2)))
            continue;  // block-uniform
        if (threadIdx.x == 0) {
            fence_async_smem();  // earlier triangles' reads of s_key (all past the last barrier)
            mbar_arrive_expect(&s_bar, (aw + bw + cw) * 8u);
            bulk_to_smem(s_key, A.key + (A.b - ao), aw * 8u, &s_bar);
            bulk_to_smem(s_key + aw, B.key + (B.b - bo), bw * 8u, &s_bar);
            if (cw) bulk_to_smem(s_ck, C.key + (C.b - co), cw * 8u, &s_bar);
        }
        if (!mbar_wait(&s_bar, bar_phase, 1u << 24)) {
            // the copy did not arrive: report it and stop using shared memory
            if (threadIdx.x == 0) atomicOr(flag, FLAG_TIMEOUT);
            mbar_wait(&s_bar, bar_phase, 1u << 24);
            return;
        }
        bar_phase ^= 1u;
        const int64_t *sA = s_key + ao, *sB = s_key + aw + bo, *sC = s_ck + co;
        // C's effective direction-0 prefix, when staged (contiguous runs
        // per thread, one block scan)
        if (c_staged) {
            const uint32_t cper = (C.n + HEAVY_THREADS - 1) / HEAVY_THREADS;
            const uint32_t cbeg = min(C.n, threadIdx.x * cper), cend = min(C.n, cbeg + cper);
            uint32_t c0 = 0;
            for (uint32_t i = cbeg; i < cend; i++) c0 += ((uint32_t)(sC[i] & 1) ^ C.flip) == 0;
            uint32_t crun = block_excl_scan_u32(c0, s_tmp);
            for (uint32_t i = cbeg; i < cend; i++) {
                s_cd0[i] = crun;
                crun += ((uint32_t)(sC[i] & 1) ^ C.flip) == 0;
            }
            if (threadIdx.x == 0) s_cd0[C.n] = s_tmp[HEAVY_WARPS];
            __syncthreads();  // s_tmp is reused below
        }
        const SList Cs{sC, s_cd0, C.n, 0u};
        auto key_at = [&](uint32_t i) { return i < na ? sA[i] : sB[i - na]; };
        // the effective direction-0 prefix over A ++ B: each thread scans a
        // contiguous run of the staged keys
        const uint32_t per = (ne + HEAVY_THREADS - 1) / HEAVY_THREADS;
        const uint32_t beg = min(ne, threadIdx.x * per), end = min(ne, beg + per);
        uint32_t cnt0 = 0;
        for (uint32_t i = beg; i < end; i++) cnt0 += ((uint32_t)(key_at(i) & 1) ^ (i < na ? A.flip : B.flip)) == 0;
        uint32_t run = block_excl_scan_u32(cnt0, s_tmp);
        for (uint32_t i = beg; i < end; i++) {
            s_d0[i] = run;
            run += ((uint32_t)(key_at(i) & 1) ^ (i < na ? A.flip : B.flip)) == 0;
        }
        if (threadIdx.x == 0) s_d0[ne] = s_tmp[HEAVY_WARPS];
        __syncthreads();
        const uint32_t a0 = s_d0[na], b0 = s_d0[ne] - a0;
        // first prefix entry of each own-direction segment: A0, A1, B0, B1
        const uint32_t sbase[4] = {0, a0 + 1, na + 2, na + 2 + b0 + 1};
        const uint32_t slen[4] = {a0, na - a0, b0, nb - b0};
        // the two-pointer form (block-uniform): each thread takes its
        // contiguous run beg .. end of A ++ B; otherwise the edges are dealt
        // out thread-strided and every bound is binary-searched
        const bool walk = merge && c_staged && C.n <= ne;
        const uint32_t e_first = walk ? beg : threadIdx.x, e_last = walk ? end : ne;
        const uint32_t e_step = walk ? 1u : (uint32_t)HEAVY_THREADS;
        for (uint32_t q = 0; q < (MODE == 1 ? nq : 1u); q++) {
            const Query Q = load_query(dq, MODE == 0 ? g : q);
            // phase 1 (and the zero entry of each segment)
            if (threadIdx.x < 32) s_pre[(threadIdx.x >> 2) * ES + sbase[threadIdx.x & 3]] = 0;
            Cursor<4> c1{};
            Cursor<3> c1h{};
            for (uint32_t e = e_first; e < e_last; e += e_step) {
                const uint32_t z = e >= na;
                if (e == na) c1.valid = c1h.valid = false;  // B's list: its bounds start over
                const uint32_t j = z ? e - na : e;
                const int64_t ke = key_at(e);
                const uint32_t de = (uint32_t)(ke & 1) ^ (z ? B.flip : A.flip);
                const uint32_t dz0 = z ? s_d0[e] - a0 : s_d0[e];
                const uint32_t rank = de ? j - dz0 : dz0;
                uint32_t v[8];
                const uint32_t at = sbase[2 * z + de] + rank + 1;
                if (q == 0) {
                    if (c_staged) phase1_values(Cs, f, Q, ke, v, walk ? &c1 : nullptr);
                    else phase1_values(C, f, Q, ke, v);
#pragma unroll
                    for (int s = 0; s < 8; s++) s_pre[s * ES + at] = v[s];
                } else {  // L(e) and its prefix sums are the first query's
                    if (c_staged) phase1_values_hrm(Cs, f, Q, ke, v, walk ? &c1h : nullptr);
                    else phase1_values_hrm(C, f, Q, ke, v);
#pragma unroll
                    for (int s = 0; s < 8; s++)
                        if (s != 2 && s != 3) s_pre[s * ES + at] = v[s];
                }
            }
            __syncthreads();
            // inclusive scans: 4 segments x 8 slots, one warp per (segment, slot)
            // (slots 2 and 3, L(e), only for the first query)
            for (uint32_t p = threadIdx.x >> 5; p < 32; p += HEAVY_WARPS) {
                const uint32_t seg = p & 3, s = p >> 2, lane = threadIdx.x & 31;
                if (q > 0 && (s == 2 || s == 3)) continue;  // warp-uniform
                P *base = s_pre + s * ES + sbase[seg] + 1;
                P carry = 0;
                for (uint32_t c0 = 0; c0 < slen[seg]; c0 += 32) {
                    const uint32_t i = c0 + lane;
                    P x = i < slen[seg] ? base[i] : P(0);
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const P y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= (uint32_t)o) x += y;
                    }
                    x += carry;
                    if (i < slen[seg]) base[i] = x;
                    carry = __shfl_sync(0xffffffffu, x, 31);
                }
            }
            __syncthreads();
            // phase 2
            Cursor<4> cc{};
            Cursor<8> co{};
            for (uint32_t e = e_first; e < e_last; e += e_step) {
                const uint32_t z = e >= na;
                if (e == na) cc.valid = co.valid = false;  // e moves to B, O to A: bounds start over
                const int64_t ke = key_at(e);
                const uint32_t de = (uint32_t)(ke & 1) ^ (z ? B.flip : A.flip);
                // O = the other list, staged: keys and its own dir-0 prefix
                const SList O = z ? SList{sA, s_d0, na, 0u} : SList{sB, s_d0 + na, nb, a0};
                const uint32_t oz = 1 - z;
                auto pref = [&](uint32_t dO, int s, uint32_t c) -> unsigned long long {
                    return (unsigned long long)s_pre[s * ES + sbase[2 * oz + dO] + c];
                };
                auto add = [&](uint32_t dO, uint32_t dC, int pia, int pib, unsigned long long n) {
                    if (!n) return;
                    const uint32_t dA = z ? dO : de, dB = z ? de : dO;
                    const int type = type_of(z ? pib : pia, dA, dB, dC);
                    if constexpr (MODE == 0) add_wide32(s_acc[type][threadIdx.x], n, &s_wide[type], ovf);
                    else if constexpr (MODE == 1) shared_add(&s_tail[q * 8 + type], n, ovf);
                    else atomicAdd(out + 8 * h + type, n);
                };
                if (c_staged) phase2_edge(O, Cs, f, Q, ke, pref, add, walk ? &cc : nullptr, walk ? &co : nullptr);
                else phase2_edge(O, C, f, Q, ke, pref, add);
            }
            __syncthreads();
        }
    }
    if constexpr (MODE == 0) {
        if (cur_g != 0xffffffffu) warp_flush32(s_acc, s_wide, out + 8 * cur_g, flag, ovf);
    }
    if constexpr (MODE == 1) block_flush(s_tail, nq * 8, out, flag, ovf);
}

// ---------------------------------------------------------------- heavy: one warp per triangle
// Heavy triangles with at most WCAP edges in A plus B: the same two phases
// as the CTA kernel, but each warp owns one triangle (and its slice of
// shared memory), so many small heavy triangles run side by side.
template <typename P>
struct WarpCap {
    static constexpr uint32_t CAP = sizeof(P) == 4 ? 128 : 64;
    static constexpr uint32_t ES = CAP + 4;
    static constexpr uint32_t CC = 256;  // C lists up to this long are staged too
    static constexpr size_t KEYS = (size_t)CAP * 8;
    static constexpr size_t D0 = ((size_t)CAP + 8) * 4;
    static constexpr size_t PRE = 8 * (size_t)ES * sizeof(P);
    static constexpr size_t CKEYS = (size_t)CC * 8;
    static constexpr size_t CD0 = ((size_t)CC + 8) * 4;
    static constexpr size_t PER_WARP = KEYS + D0 + PRE + CKEYS + CD0;
    static constexpr size_t bytes(int mode, uint32_t nq) {
        return HEAVY_WARPS * PER_WARP + (mode == 1 ? (size_t)nq * 64 : mode == 0 ? 8 * 256 * 8 : 0);
    }
};

template <typename P, int MODE, bool ST>
__global__ void __launch_bounds__(HEAVY_THREADS)
    heavy_warp_kernel(const GraphView *__restrict__ gvs, const uint64_t *__restrict__ hw_pre, uint32_t G,
                      const int64_t *dq, uint32_t nq, unsigned long long *out, unsigned long long *flag,
                      const uint64_t *idx, uint64_t nidx) {
    using Cap = WarpCap<P>;
    constexpr uint32_t ES = Cap::ES;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *mine = smem + w * Cap::PER_WARP;
    int64_t *s_key = reinterpret_cast<int64_t *>(mine);
    uint32_t *s_d0 = reinterpret_cast<uint32_t *>(mine + Cap::KEYS);
    P *s_pre = reinterpret_cast<P *>(mine + Cap::KEYS + Cap::D0);
    int64_t *s_ck = reinterpret_cast<int64_t *>(mine + Cap::KEYS + Cap::D0 + Cap::PRE);
    uint32_t *s_cd0 = reinterpret_cast<uint32_t *>(mine + Cap::KEYS + Cap::D0 + Cap::PRE + Cap::CKEYS);
    unsigned long long *s_tail = reinterpret_cast<unsigned long long *>(smem + HEAVY_WARPS * Cap::PER_WARP);
    auto s_acc = reinterpret_cast<unsigned long long (*)[256]>(s_tail);  // MODE 0
    if constexpr (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
    }
    if constexpr (MODE == 1) {
        for (uint32_t i = threadIdx.x; i < nq * 8; i += blockDim.x) s_tail[i] = 0;
        __syncthreads();
    }
    unsigned ovf = 0;
    uint32_t cur_g = 0xffffffffu;
    const uint64_t nitems = MODE == 2 ? nidx : __ldg(hw_pre + G);
    const uint64_t gw = (uint64_t)blockIdx.x * HEAVY_WARPS + w, nw = (uint64_t)gridDim.x * HEAVY_WARPS;
    for (uint64_t h = gw; h < nitems; h += nw) {
        const uint32_t g = MODE == 0 ? graph_of(hw_pre, G, h) : 0u;
        if constexpr (MODE == 0) {
            if (g != cur_g) {
                if (cur_g != 0xffffffffu) warp_flush(s_acc, out + 8 * cur_g, flag, ovf);
                cur_g = g;
            }
        }
        const GraphView &gv = gvs[g];
        if ((sizeof(P) == 8) != (gv.wide != 0)) continue;  // the other width's launch takes it
        const KeyFmt f{gv.shift, gv.span, ST};
        const uint64_t hl = MODE == 2 ? idx[h] : (MODE == 0 ? h - __ldg(hw_pre + g) : h);
        const uint4 r = __ldg(gv.tri + gv.n_light + hl);
        const GList A = glist(gv, r.x, r.w & TriRec::FLIP_A);
        const GList B = glist(gv, r.y, (r.w & TriRec::FLIP_B) ? 1u : 0u);
        const GList C = glist(gv, r.z, (r.w & TriRec::FLIP_C) ? 1u : 0u);
        const uint32_t na = A.n, nb = B.n, ne = na + nb;
        // stage A ++ B and the effective direction-0 prefix over it
        uint32_t carry = 0;
        for (uint32_t c0 = 0; c0 < ne; c0 += 32) {
            const uint32_t i = c0 + lane;
            uint32_t is0 = 0;
            if (i < ne) {
                const int64_t k = i < na ? __ldg(A.key + A.b + i) : __ldg(B.key + B.b + (i - na));
                s_key[i] = k;
                is0 = ((uint32_t)(k & 1) ^ (i < na ? A.flip : B.flip)) == 0;
            }
            uint32_t x = is0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (i < ne) s_d0[i] = carry + x - is0;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) s_d0[ne] = carry;
        // a short C list is staged as well (keys and effective dir-0
        // prefix), so both phases search it in shared memory; a longer one
        // is searched where it lies
        const bool c_staged = C.n <= Cap::CC;  // warp-uniform
        if (c_staged) {
            uint32_t cc = 0;
            for (uint32_t c0 = 0; c0 < C.n; c0 += 32) {
                const uint32_t i = c0 + lane;
                uint32_t is0 = 0;
                if (i < C.n) {
                    const int64_t k = __ldg(C.key + C.b + i);
                    s_ck[i] = k;
                    is0 = ((uint32_t)(k & 1) ^ C.flip) == 0;
                }
                uint32_t x = is0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= (uint32_t)o) x += y;
                }
                if (i < C.n) s_cd0[i] = cc + x - is0;
                cc += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) s_cd0[C.n] = cc;
        }
        __syncwarp();
        const uint32_t a0 = s_d0[na], b0 = carry - a0;
        const uint32_t sbase[4] = {0, a0 + 1, na + 2, na + 2 + b0 + 1};
        const uint32_t slen[4] = {a0, na - a0, b0, nb - b0};
        const SList Cs{s_ck, s_cd0, C.n, 0u};
        for (uint32_t q = 0; q < (MODE == 1 ? nq : 1u); q++) {
            const Query Q = load_query(dq, MODE == 0 ? g : q);
            // phase 1 (and the zero entry of each segment)
            s_pre[(lane >> 2) * ES + sbase[lane & 3]] = 0;
            for (uint32_t e = lane; e < ne; e += 32) {
                const uint32_t z = e >= na;
                const uint32_t j = z ? e - na : e;
                const int64_t ke = s_key[e];
                const uint32_t de = (uint32_t)(ke & 1) ^ (z ? B.flip : A.flip);
                const uint32_t dz0 = z ? s_d0[e] - a0 : s_d0[e];
                const uint32_t rank = de ? j - dz0 : dz0;
                uint32_t v[8];
                const uint32_t at = sbase[2 * z + de] + rank + 1;
                if (q == 0) {
                    if (c_staged) phase1_values(Cs, f, Q, ke, v);
                    else phase1_values(C, f, Q, ke, v);
#pragma unroll
                    for (int s = 0; s < 8; s++) s_pre[s * ES + at] = v[s];
                } else {  // L(e) and its prefix sums are the first query's
                    if (c_staged) phase1_values_hrm(Cs, f, Q, ke, v);
                    else phase1_values_hrm(C, f, Q, ke, v);
#pragma unroll
                    for (int s = 0; s < 8; s++)
                        if (s != 2 && s != 3) s_pre[s * ES + at] = v[s];
                }
            }
            __syncwarp();
            {  // inclusive scans: lane p scans (segment p & 3, slot p >> 2);
               // slots 2 and 3, L(e), only for the first query
                const uint32_t seg = lane & 3, s = lane >> 2;
                if (q == 0 || (s != 2 && s != 3)) {
                    P *base = s_pre + s * ES + sbase[seg] + 1;
                    P run = 0;
                    for (uint32_t i = 0; i < slen[seg]; i++) {
                        run += base[i];
                        base[i] = run;
                    }
                }
            }
            __syncwarp();
            // phase 2
            for (uint32_t e = lane; e < ne; e += 32) {
                const uint32_t z = e >= na;
                const int64_t ke = s_key[e];
                const uint32_t de = (uint32_t)(ke & 1) ^ (z ? B.flip : A.flip);
                const SList O = z ? SList{s_key, s_d0, na, 0u} : SList{s_key + na, s_d0 + na, nb, a0};
                const uint32_t oz = 1 - z;
                auto pref = [&](uint32_t dO, int s, uint32_t c) -> unsigned long long {
                    return (unsigned long long)s_pre[s * ES + sbase[2 * oz + dO] + c];
                };
                auto add = [&](uint32_t dO, uint32_t dC, int pia, int pib, unsigned long long n) {
                    if (!n) return;
                    const uint32_t dA = z ? dO : de, dB = z ? de : dO;
                    const int type = type_of(z ? pib : pia, dA, dB, dC);
                    if constexpr (MODE == 0) add_checked(s_acc[type][threadIdx.x], n, ovf);
                    else if constexpr (MODE == 1) shared_add(&s_tail[q * 8 + type], n, ovf);
                    else atomicAdd(out + 8 * h + type, n);
                };
                if (c_staged) phase2_edge(O, Cs, f, Q, ke, pref, add);
                else phase2_edge(O, C, f, Q, ke, pref, add);
            }
            __syncwarp();
        }
    }
    if constexpr (MODE == 0) {
        if (cur_g != 0xffffffffu) warp_flush(s_acc, out + 8 * cur_g, flag, ovf);
    }
    if constexpr (MODE == 1) block_flush(s_tail, nq * 8, out, flag, ovf);
}

// ---------------------------------------------------------------- huge: flat path
struct HugeArgs {
    GraphView gv;
    const uint4 *__restrict__ tri;      // huge records
    const uint64_t *__restrict__ eoff;  // [nh + 1] enumerated-edge offsets
    uint64_t nh, total;
    void *pre;                          // prefix entries: 8 values each
    unsigned long long *per_tri;        // sample mode: per-record outputs
    // queries of one pass: query q's prefix entries start at entry
    // q * qstride (qstride = total + 4 nh) and its counts at out + 8 q
    uint32_t nq = 1;
    uint64_t qstride = 0;
};

// Scratch one batched pass of the flat path may take for its queries'
// prefix entries (a single query always gets its own).
constexpr size_t HUGE_PASS_BYTES = size_t(64) << 20;

// Locates enumerated edge e: the last triangle h with eoff[h] <= e.
__device__ __forceinline__ uint64_t find_tri(const uint64_t *__restrict__ eoff, uint64_t nh, uint64_t e) {
    uint64_t lo = 0, hi = nh;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldg(eoff + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

struct HugeTri {
    GList A, B, C;
    uint32_t a0, b0;  // effective direction-0 counts of A and B
    uint64_t base;    // first prefix entry of this triangle
};

__device__ __forceinline__ HugeTri huge_tri(const HugeArgs &a, uint64_t h) {
    const uint4 r = __ldg(a.tri + h);
    HugeTri t;
    t.A = glist(a.gv, r.x, r.w & TriRec::FLIP_A);
    t.B = glist(a.gv, r.y, (r.w & TriRec::FLIP_B) ? 1u : 0u);
    t.C = glist(a.gv, r.z, (r.w & TriRec::FLIP_C) ? 1u : 0u);
    t.a0 = t.A.d0(t.A.n);
    t.b0 = t.B.d0(t.B.n);
    t.base = __ldg(a.eoff + h) + 4 * h;
    return t;
}

// first prefix entry of the own-direction-d segment of list Z (0 = A, 1 = B)
__device__ __forceinline__ uint64_t seg_base(const HugeTri &t, uint32_t z, uint32_t d) {
    uint64_t b = t.base;
    if (z) b += t.A.n + 2;
    const uint32_t n0 = z ? t.b0 : t.a0;
    if (d) b += n0 + 1;
    return b;
}

template <typename P, bool ST>
__global__ void __launch_bounds__(HEAVY_THREADS) huge_phase1(HugeArgs a, const int64_t *dq) {
    const KeyFmt f{a.gv.shift, a.gv.span, ST};
    // over (enumerated edge, query) of the pass
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.total * a.nq;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t qi = (uint32_t)(x / a.total);
        const uint64_t e = x - (uint64_t)qi * a.total;
        const Query q = load_query(dq, qi);
        P *pre = static_cast<P *>(a.pre) + 8 * a.qstride * qi;
        const uint64_t h = find_tri(a.eoff, a.nh, e);
        const HugeTri t = huge_tri(a, h);
        uint32_t j = (uint32_t)(e - __ldg(a.eoff + h));
        const uint32_t z = j >= t.A.n;
        const GList &Z = z ? t.B : t.A;
        if (z) j -= t.A.n;
        const int64_t ke = __ldg(Z.key + Z.b + j);
        const uint32_t d = (uint32_t)(ke & 1) ^ Z.flip;
        const uint32_t z0 = Z.d0(j);
        const uint32_t rank = d ? j - z0 : z0;
        uint32_t v[8];
        phase1_values(t.C, f, q, ke, v);
        P *o = pre + 8 * (seg_base(t, z, d) + rank + 1);
#pragma unroll
        for (int s = 0; s < 8; s++) o[s] = v[s];
    }
}

// Inclusive scan of each own-direction segment (entry 0 of a segment is 0).
// One warp per segment; 4 segments per huge triangle.
template <typename P>
__global__ void __launch_bounds__(HEAVY_THREADS) huge_scan(HugeArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t x = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < 4 * a.nh * a.nq;
         x += warps) {
        const uint32_t qi = (uint32_t)(x / (4 * a.nh));
        const uint64_t sidx = x - (uint64_t)qi * 4 * a.nh;
        P *pre = static_cast<P *>(a.pre) + 8 * a.qstride * qi;
        const uint64_t h = sidx >> 2;
        const uint32_t z = (uint32_t)((sidx >> 1) & 1);
        const uint32_t d = (uint32_t)(sidx & 1);
        const HugeTri t = huge_tri(a, h);
        const uint32_t nz = z ? t.B.n : t.A.n, n0 = z ? t.b0 : t.a0;
        const uint32_t len = d ? nz - n0 : n0;
        P *seg = pre + 8 * seg_base(t, z, d);
        if (lane < 8) seg[lane] = 0;
        P carry[8];
#pragma unroll
        for (int s = 0; s < 8; s++) carry[s] = 0;
        for (uint32_t c = 0; c < len; c += 32) {
            const uint32_t i = c + lane;
            P v[8];
#pragma unroll
            for (int s = 0; s < 8; s++) v[s] = i < len ? seg[8 * (i + 1) + s] : P(0);
#pragma unroll
            for (int s = 0; s < 8; s++) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const P y = __shfl_up_sync(0xffffffffu, v[s], o);
                    if (lane >= (uint32_t)o) v[s] += y;
                }
                v[s] += carry[s];
                carry[s] = __shfl_sync(0xffffffffu, v[s], 31);
            }
            if (i < len) {
#pragma unroll
                for (int s = 0; s < 8; s++) seg[8 * (i + 1) + s] = v[s];
            }
        }
    }
}

template <typename P, bool ST>
__global__ void __launch_bounds__(HEAVY_THREADS)
    huge_phase2(HugeArgs a, const int64_t *dq, unsigned long long *out, unsigned long long *flag) {
    __shared__ unsigned long long s_acc[8][256];
#pragma unroll
    for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
    unsigned ovf = 0;
    const KeyFmt f{a.gv.shift, a.gv.span, ST};
    if (a.nq > 1) {
        // several queries: over (enumerated edge, query), each count added
        // to its query's row with a carry-checked device atomic
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.total * a.nq;
             x += (uint64_t)gridDim.x * blockDim.x) {
            const uint32_t qi = (uint32_t)(x / a.total);
            const uint64_t e = x - (uint64_t)qi * a.total;
            const Query q = load_query(dq, qi);
            const P *pre = static_cast<const P *>(a.pre) + 8 * a.qstride * qi;
            const uint64_t h = find_tri(a.eoff, a.nh, e);
            const HugeTri t = huge_tri(a, h);
            uint32_t j = (uint32_t)(e - __ldg(a.eoff + h));
            const uint32_t z = j >= t.A.n;
            if (z) j -= t.A.n;
            const GList &Z = z ? t.B : t.A;
            const GList &O = z ? t.A : t.B;
            const uint32_t oz = 1 - z;
            const int64_t ke = __ldg(Z.key + Z.b + j);
            const uint32_t de = (uint32_t)(ke & 1) ^ Z.flip;
            auto pref = [&](uint32_t dO, int s, uint32_t c) -> unsigned long long {
                return (unsigned long long)pre[8 * (seg_base(t, oz, dO) + c) + s];
            };
            auto add = [&](uint32_t dO, uint32_t dC, int pia, int pib, unsigned long long n) {
                if (!n) return;
                const uint32_t dA = z ? dO : de, dB = z ? de : dO;
                const int type = type_of(z ? pib : pia, dA, dB, dC);
                const unsigned long long old = atomicAdd(out + 8 * (size_t)qi + type, n);
                if (old + n < old) ovf = 1;
            };
            phase2_edge(O, t.C, f, q, ke, pref, add);
        }
        if (ovf) atomicOr(flag, 1ull);
        return;
    }
    const Query q = load_query(dq, 0);
    const P *pre = static_cast<const P *>(a.pre);
    const uint64_t iters = (a.total + (uint64_t)gridDim.x * blockDim.x - 1) / ((uint64_t)gridDim.x * blockDim.x);
    for (uint64_t it = 0; it < iters; it++) {  // uniform trip count (warp_flush needs full warps)
        const uint64_t e = (it * gridDim.x + blockIdx.x) * (uint64_t)blockDim.x + threadIdx.x;
        if (e >= a.total) continue;
        const uint64_t h = find_tri(a.eoff, a.nh, e);
        const HugeTri t = huge_tri(a, h);
        uint32_t j = (uint32_t)(e - __ldg(a.eoff + h));
        const uint32_t z = j >= t.A.n;  // this edge's list Z (0 = A, 1 = B); O is the other
        if (z) j -= t.A.n;
        const GList &Z = z ? t.B : t.A;
        const GList &O = z ? t.A : t.B;
        const uint32_t oz = 1 - z;
        const int64_t ke = __ldg(Z.key + Z.b + j);
        const uint32_t de = (uint32_t)(ke & 1) ^ Z.flip;
        unsigned long long *pt = a.per_tri ? a.per_tri + 8 * h : nullptr;
        auto pref = [&](uint32_t dO, int s, uint32_t c) -> unsigned long long {
            return (unsigned long long)pre[8 * (seg_base(t, oz, dO) + c) + s];
        };
        auto add = [&](uint32_t dO, uint32_t dC, int pia, int pib, unsigned long long n) {
            if (!n) return;
            const uint32_t dA = z ? dO : de, dB = z ? de : dO;
            const int type = type_of(z ? pib : pia, dA, dB, dC);
            if (pt) atomicAdd(pt + type, n);
            else add_checked(s_acc[type][threadIdx.x], n, ovf);
        };
        phase2_edge(O, t.C, f, q, ke, pref, add);
    }
    if (!a.per_tri) warp_flush(s_acc, out, flag, ovf);
}

template <typename P>
void run_huge(ttc_graph *g, const HugeArgs &ha, const int64_t *dq_one, unsigned long long *out,
              unsigned long long *flag, cudaStream_t s) {
    if (!ha.nh) return;
    const unsigned grid = (unsigned)(sm_count() * 8);
    prof_begin(g, s, "huge_phase1");
    if (ha.gv.strict) huge_phase1<P, true><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one);
    else huge_phase1<P, false><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
    prof_begin(g, s, "huge_scan");
    huge_scan<P><<<grid, HEAVY_THREADS, 0, s>>>(ha);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
    prof_begin(g, s, "huge_phase2");
    if (ha.gv.strict) huge_phase2<P, true><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one, out, flag);
    else huge_phase2<P, false><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one, out, flag);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
}

HugeArgs huge_args(ttc_graph *g, void *scratch) {
    HugeArgs ha{};
    ha.gv = g->view_host;
    // (a streamed handle lists no light records: the view's light count is 0)
    ha.tri = g->tri.get() + g->view_host.n_light + g->st.tau_hwarp + g->st.tau_hcta;
    ha.eoff = g->huge_eoff.get();
    ha.nh = g->st.tau_huge;
    ha.total = g->huge_elems;
    ha.pre = scratch;
    return ha;
}

// Persistent grids: at most `per_sm` CTAs per SM, never more than the work.
unsigned light_grid(uint64_t chunks, int per_sm = 8) {
    const uint64_t want = (chunks + LIGHT_WARPS - 1) / LIGHT_WARPS;
    const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
    return (unsigned)(want < 1 ? 1 : want < cap ? want : cap);
}

unsigned heavy_grid(uint64_t items, int per_sm = 2) {
    const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
    return (unsigned)(items < 1 ? 1 : items < cap ? items : cap);
}

template <typename P, int MODE, bool ST>
void launch_fused(const GraphView *gvs, const uint64_t *heavy_pre, uint32_t G, uint64_t items, const int64_t *dq,
                  uint32_t nq, unsigned long long *out, unsigned long long *flag, const uint64_t *idx,
                  uint64_t nidx, cudaStream_t s, int per_sm, uint32_t merge) {
    ensure_smem((const void *)heavy_fused_kernel<P, MODE, ST>, FusedCap<P>::bytes(1, MAX_BATCH_SMEM_Q));
    heavy_fused_kernel<P, MODE, ST><<<heavy_grid(items, per_sm), HEAVY_THREADS, FusedCap<P>::bytes(MODE, nq), s>>>(
        gvs, heavy_pre, G, dq, nq, out, flag, idx, nidx, merge);
    TTC_LAUNCH_CHECK();
}

template <typename P, int MODE, bool ST>
void launch_warp(const GraphView *gvs, const uint64_t *hw_pre, uint32_t G, uint64_t items, const int64_t *dq,
                 uint32_t nq, unsigned long long *out, unsigned long long *flag, const uint64_t *idx, uint64_t nidx,
                 cudaStream_t s, int per_sm = 4) {
    ensure_smem((const void *)heavy_warp_kernel<P, MODE, ST>, WarpCap<P>::bytes(1, MAX_BATCH_SMEM_Q));
    const uint64_t want = (items + HEAVY_WARPS - 1) / HEAVY_WARPS;
    const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
    const unsigned grid = (unsigned)(want < 1 ? 1 : want < cap ? want : cap);
    heavy_warp_kernel<P, MODE, ST><<<grid, HEAVY_THREADS, WarpCap<P>::bytes(MODE, nq), s>>>(gvs, hw_pre, G, dq, nq, out,
                                                                                       flag, idx, nidx);
    TTC_LAUNCH_CHECK();
}

// kind: bit 0 = 64-bit prefix sums (wide lists), bit 1 = strict time order,
// bit 2 = the one-CTA class takes the two-pointer form where it applies
inline int heavy_kind(int wide, bool strict, bool merge = false) {
    return (wide ? 1 : 0) | (strict ? 2 : 0) | (merge ? 4 : 0);
}

template <int MODE>
void launch_warp_any(int kind, const GraphView *gvs, const uint64_t *hw_pre, uint32_t G, uint64_t items,
                     const int64_t *dq, uint32_t nq, unsigned long long *out, unsigned long long *flag,
                     const uint64_t *idx, uint64_t nidx, cudaStream_t s, int per_sm = 4) {
    switch (kind & 3) {
        case 0: launch_warp<uint32_t, MODE, false>(gvs, hw_pre, G, items, dq, nq, out, flag, idx, nidx, s, per_sm); break;
        case 1: launch_warp<unsigned long long, MODE, false>(gvs, hw_pre, G, items, dq, nq, out, flag, idx, nidx, s,
                                                            per_sm); break;
        case 2: launch_warp<uint32_t, MODE, true>(gvs, hw_pre, G, items, dq, nq, out, flag, idx, nidx, s, per_sm); break;
        default: launch_warp<unsigned long long, MODE, true>(gvs, hw_pre, G, items, dq, nq, out, flag, idx, nidx, s,
                                                             per_sm);
    }
}

template <int MODE>
void launch_fused_any(int kind, const GraphView *gvs, const uint64_t *heavy_pre, uint32_t G, uint64_t items,
                      const int64_t *dq, uint32_t nq, unsigned long long *out, unsigned long long *flag,
                      const uint64_t *idx, uint64_t nidx, cudaStream_t s, int per_sm = 2) {
    const uint32_t merge = (kind & 4) ? 1u : 0u;
    switch (kind & 3) {
        case 0: launch_fused<uint32_t, MODE, false>(gvs, heavy_pre, G, items, dq, nq, out, flag, idx, nidx, s, per_sm,
                                                    merge); break;
        case 1: launch_fused<unsigned long long, MODE, false>(gvs, heavy_pre, G, items, dq, nq, out, flag, idx, nidx, s,
                                                              per_sm, merge); break;
        case 2: launch_fused<uint32_t, MODE, true>(gvs, heavy_pre, G, items, dq, nq, out, flag, idx, nidx, s, per_sm,
                                                   merge); break;
        default: launch_fused<unsigned long long, MODE, true>(gvs, heavy_pre, G, items, dq, nq, out, flag, idx, nidx, s,
                                                              per_sm, merge);
    }
}

// The record ranges one count covers: per bin a device graph view and the
// prefix its kernel reads, and the huge records as flat-path arguments.  The
// whole graph uses the handle's own view; a shard uses views whose record
// pointer starts at the shard's first record of each bin.
struct BinViews {
    const GraphView *light_view, *hw_view, *hc_view;
    const uint64_t *light_pre, *hw_pre, *hc_pre;  // {0, 32-record chunks}, {0, n_hw}, {0, n_hc}
    uint64_t n_light, n_hw, n_hc;
    HugeArgs huge;                                 // huge.nh = 0: none
    uint32_t huge_qcap = 1;                        // queries one pass of the flat path takes
};

// One query (acc[8] + flag) or a batch of k (acc[k][8] + flag at acc[8 k])
// over the records of `b`; the huge path's prefix arrays live in `scratch`.
void count_bins(ttc_graph *g, const BinViews &b, const int64_t *dq, uint32_t k, unsigned long long *acc,
                cudaStream_t s0) {
    unsigned long long *flag = acc + 8 * (size_t)k;
    // the heavy bins (few triangles, few CTAs) run on the side stream beside
    // the light bin on the count's stream; every kernel adds into acc with
    // atomics, and the side stream is joined back before the count ends.
    // The light kernel is launched first, so its CTAs take the SMs and the
    // heavy CTAs fill the slots its last wave leaves (measured on the
    // power-law workload: unbounded query 7.73 -> 7.44 ms, the step's batch
    // 8.14 -> 7.72 ms; launching the heavy bins first cost the single query)
    const bool fork = (b.n_hw || b.n_hc || b.huge.nh) && (b.n_light || g->streamed);
    cudaStream_t s = s0;
    if (fork) {
        if (!g->side) {
            TTC_CUDA(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
            TTC_CUDA(cudaEventCreateWithFlags(&g->side_fork, cudaEventDisableTiming));
            TTC_CUDA(cudaEventCreateWithFlags(&g->side_join, cudaEventDisableTiming));
        }
        TTC_CUDA(cudaEventRecord(g->side_fork, s0));
        TTC_CUDA(cudaStreamWaitEvent(g->side, g->side_fork, 0));
        s = g->side;
    }
    if (g->streamed) stream_count_light(g, dq, k, acc, s0);  // the light triangles are found again and counted
    else if (b.n_light) count_light_records(g, b.light_view, b.light_pre, b.n_light, dq, k, acc, s0);
    const uint64_t nw = b.n_hw, nc = b.n_hc;
    for (uint32_t q0 = 0; q0 < k && (nw || nc); q0 += MAX_BATCH_SMEM_Q) {
        const uint32_t nq = k - q0 < MAX_BATCH_SMEM_Q ? k - q0 : MAX_BATCH_SMEM_Q;
        const int mode = k == 1 ? 0 : 1;
        if (nw) {
            prof_begin(g, s, mode ? "heavy_warp_batch" : "heavy_warp");
            if (mode) launch_warp_any<1>(heavy_kind(g->heavy_wide, g->strict), b.hw_view, b.hw_pre, 1, nw,
                                         dq + 3 * (size_t)q0, nq, acc + 8 * (size_t)q0, flag, nullptr, 0, s);
            else launch_warp_any<0>(heavy_kind(g->heavy_wide, g->strict), b.hw_view, b.hw_pre, 1, nw, dq, 1, acc,
                                    flag, nullptr, 0, s);
            prof_end(g, s);
        }
        if (nc) {
            prof_begin(g, s, mode ? "heavy_cta_batch" : "heavy_cta");
            const int kc = heavy_kind(g->heavy_wide, g->strict, g->st.heavy_merge == TTC_HEAVY_MERGE);
            if (mode) launch_fused_any<1>(kc, b.hc_view, b.hc_pre, 1, nc, dq + 3 * (size_t)q0, nq, acc + 8 * (size_t)q0,
                                          flag, nullptr, 0, s);
            else launch_fused_any<0>(kc, b.hc_view, b.hc_pre, 1, nc, dq, 1, acc, flag, nullptr, 0, s);
            prof_end(g, s);
        }
    }
    if (b.huge.nh) {
        // the flat path in passes of up to huge_qcap queries (one launch per
        // phase each; the scratch holds that many queries' prefix entries)
        for (uint32_t q0 = 0; q0 < k; q0 += b.huge_qcap) {
            HugeArgs ha = b.huge;
            ha.nq = std::min(b.huge_qcap, k - q0);
            ha.qstride = ha.total + 4 * ha.nh;
            if (g->heavy_wide) run_huge<unsigned long long>(g, ha, dq + 3 * (size_t)q0, acc + 8 * (size_t)q0, flag, s);
            else run_huge<uint32_t>(g, ha, dq + 3 * (size_t)q0, acc + 8 * (size_t)q0, flag, s);
        }
    }
    if (fork) {
        TTC_CUDA(cudaEventRecord(g->side_join, g->side));
        TTC_CUDA(cudaStreamWaitEvent(s0, g->side_join, 0));
    }
}

void count_graph(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, void *scratch,
                 cudaStream_t s) {
    if (!g->st.tau || !k) return;
    BinViews b{};
    b.light_view = b.hw_view = b.hc_view = g->view.get();
    b.light_pre = g->prefix.get();
    b.hw_pre = g->prefix.get() + 2;
    b.hc_pre = g->prefix.get() + 4;
    b.n_light = g->st.tau_light;
    b.n_hw = g->st.tau_hwarp;
    b.n_hc = g->st.tau_hcta;
    if (g->st.tau_huge) b.huge = huge_args(g, scratch);
    b.huge_qcap = huge_pass_queries(g, k);
    count_bins(g, b, dq, k, acc, s);
}

// Vertex triple (u, v, w) of each sampled record: A = {u, v}, B = {u, w}.
__global__ void record_vertices_kernel(const uint4 *tri, const uint2 *pv, const uint64_t *idx, uint64_t count,
                                       uint32_t *out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = tri[idx[i]];
        const uint2 a = pv[r.x], b = pv[r.y];
        const uint32_t u = (a.x == b.x || a.x == b.y) ? a.x : a.y;
        out[3 * i] = u;
        out[3 * i + 1] = a.x == u ? a.y : a.x;
        out[3 * i + 2] = b.x == u ? b.y : b.x;
    }
}

__global__ void record_sizes_kernel(const uint4 *tri, const uint64_t *idx, uint64_t count, const uint32_t *poff,
                                    uint4 *recs, uint64_t *sizes) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = tri[idx[i]];
        recs[i] = r;
        sizes[i] = (poff[r.x + 1] - poff[r.x]) + (poff[r.y + 1] - poff[r.y]);
    }
}

}  // namespace

void count_light_records(ttc_graph *g, const GraphView *gv, const uint64_t *light_pre, uint64_t nl,
                         const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s) {
    if (!nl || !k) return;
    unsigned long long *flag = acc + 8 * (size_t)k;
    if (k == 1) {
        prof_begin(g, s, "light");
        constexpr int R0 = LIGHT_SINGLE_R;
        const unsigned grid = light_grid((nl + 32 * R0 - 1) / (32 * R0));
        if (g->strict)
            light_kernel<0, R0, true><<<grid, LIGHT_THREADS, 0, s>>>(gv, light_pre, 1, dq, 1, acc, flag, nullptr, 0);
        else
            light_kernel<0, R0, false><<<grid, LIGHT_THREADS, 0, s>>>(gv, light_pre, 1, dq, 1, acc, flag, nullptr, 0);
        TTC_LAUNCH_CHECK();
        prof_end(g, s);
        return;
    }
    // work items of 32 * LIGHT_BATCH_R records
    const uint64_t chunks = (nl + 32 * LIGHT_BATCH_R - 1) / (32 * LIGHT_BATCH_R);
    for (uint32_t q0 = 0; q0 < k; q0 += MAX_BATCH_SMEM_Q) {
        const uint32_t nq = k - q0 < MAX_BATCH_SMEM_Q ? k - q0 : MAX_BATCH_SMEM_Q;
        // enough (chunk, query group) items to fill the GPU, and no
        // smaller groups than that: each group re-reads its chunk
        const uint64_t want_items = (uint64_t)sm_count() * 8 * LIGHT_WARPS;
        const uint32_t groups = (uint32_t)std::min<uint64_t>(nq, (want_items + chunks - 1) / chunks);
        const uint32_t qpw = (nq + groups - 1) / groups;
        prof_begin(g, s, "light_batch");
        const size_t smem = nq * 64 + (qpw <= LIGHT_QT ? (size_t)LIGHT_QT * 8 * LIGHT_THREADS * 4
                                                       : (size_t)nq * (sizeof(Query) + 4));
        {
            const size_t most = MAX_BATCH_SMEM_Q * 64 + LIGHT_QT * 8 * LIGHT_THREADS * 4;
            ensure_smem((const void *)light_kernel<1, LIGHT_BATCH_R, false>, most);
            ensure_smem((const void *)light_kernel<1, LIGHT_BATCH_R, true>, most);
        }
        const unsigned grid = light_grid(chunks * ((nq + qpw - 1) / qpw));
        if (g->strict)
            light_kernel<1, LIGHT_BATCH_R, true><<<grid, LIGHT_THREADS, smem, s>>>(
                gv, light_pre, 1, dq + 3 * (size_t)q0, nq, acc + 8 * (size_t)q0, flag, nullptr, 0, qpw);
        else
            light_kernel<1, LIGHT_BATCH_R, false><<<grid, LIGHT_THREADS, smem, s>>>(
                gv, light_pre, 1, dq + 3 * (size_t)q0, nq, acc + 8 * (size_t)q0, flag, nullptr, 0, qpw);
        TTC_LAUNCH_CHECK();
        prof_end(g, s);
    }
}

size_t heavy_scratch_bytes(const ttc_graph *g) {
    const size_t entries = (size_t)g->huge_elems + 4 * (size_t)g->st.tau_huge;
    return g->st.tau_huge ? entries * 8 * (g->heavy_wide ? 8 : 4) : 0;
}

// Queries one batched pass of the flat path takes: all k while their prefix
// entries fit HUGE_PASS_BYTES, else as many as do (at least one).
// ($TTC_HUGE_PASS_BYTES, when set, replaces the cap.)
uint32_t huge_pass_queries(const ttc_graph *g, uint32_t k) {
    const size_t one = heavy_scratch_bytes(g);
    if (k <= 1 || !one) return 1;
    const char *e = getenv("TTC_HUGE_PASS_BYTES");
    const long long v = e ? atoll(e) : 0;
    const size_t cap = v > 0 ? (size_t)v : HUGE_PASS_BYTES;
    return (uint32_t)std::min<size_t>(k, std::max<size_t>(1, cap / one));
}

void count_queue(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s) {
    void *scratch = nullptr;
    const size_t bytes = heavy_scratch_bytes(g) * huge_pass_queries(g, k);
    if (bytes) {
        if (g->scratch.count < bytes) g->scratch.alloc(bytes, s);
        scratch = g->scratch.get();
    }
    count_graph(g, dq, k, acc, scratch, s);
}

// Records [lo, hi) of a bin of n records for shard `shard` of `nshards`:
// consecutive slices of near-equal length, so the shards partition the bin.
static inline void shard_slice(uint64_t n, uint32_t shard, uint32_t nshards, uint64_t &lo, uint64_t &hi) {
    lo = (uint64_t)(((unsigned __int128)n * shard) / nshards);
    hi = (uint64_t)(((unsigned __int128)n * (shard + 1)) / nshards);
}

void count_queue_shard(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, uint32_t shard,
                       uint32_t nshards, cudaStream_t s) {
    if (!g->st.tau || !k) return;
    uint64_t lo[4], hi[4];
    shard_slice(g->st.tau_light, shard, nshards, lo[0], hi[0]);
    shard_slice(g->st.tau_hwarp, shard, nshards, lo[1], hi[1]);
    shard_slice(g->st.tau_hcta, shard, nshards, lo[2], hi[2]);
    shard_slice(g->st.tau_huge, shard, nshards, lo[3], hi[3]);
    // views whose record pointer starts at the slice: the light kernel reads
    // tri[i], the warp kernel tri[n_light + i], the CTA kernel
    // tri[n_light + n_hwarp + i] for i below the slice length
    GraphView v[3] = {g->view_host, g->view_host, g->view_host};
    v[0].tri = g->tri.get() + lo[0];
    v[0].n_light = hi[0] - lo[0];
    v[1].tri = g->tri.get() + lo[1];
    v[2].tri = g->tri.get() + lo[2];
    const uint64_t pre[6] = {0, (hi[0] - lo[0] + 31) / 32, 0, hi[1] - lo[1], 0, hi[2] - lo[2]};
    if (!g->shard_view.get()) {
        g->shard_view.alloc(3, s);
        g->shard_pre.alloc(6, s);
    }
    TTC_CUDA(cudaMemcpyAsync(g->shard_view.get(), v, sizeof v, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemcpyAsync(g->shard_pre.get(), pre, sizeof pre, cudaMemcpyHostToDevice, s));
    BinViews b{};
    b.light_view = g->shard_view.get();
    b.hw_view = g->shard_view.get() + 1;
    b.hc_view = g->shard_view.get() + 2;
    b.light_pre = g->shard_pre.get();
    b.hw_pre = g->shard_pre.get() + 2;
    b.hc_pre = g->shard_pre.get() + 4;
    b.n_light = hi[0] - lo[0];
    b.n_hw = hi[1] - lo[1];
    b.n_hc = hi[2] - lo[2];
    if (hi[3] > lo[3]) {
        // the slice's enumerated-edge offsets, rebased to start at zero
        if (g->huge_eoff_host.size() != g->st.tau_huge + 1) {
            g->huge_eoff_host.resize(g->st.tau_huge + 1);
            TTC_CUDA(cudaMemcpyAsync(g->huge_eoff_host.data(), g->huge_eoff.get(), g->huge_eoff_host.size() * 8,
                                     cudaMemcpyDeviceToHost, s));
            TTC_CUDA(cudaStreamSynchronize(s));
        }
        const uint64_t nh = hi[3] - lo[3];
        std::vector<uint64_t> eo(nh + 1);
        for (uint64_t i = 0; i <= nh; i++) eo[i] = g->huge_eoff_host[lo[3] + i] - g->huge_eoff_host[lo[3]];
        if (g->shard_eoff.count < nh + 1) g->shard_eoff.alloc(g->st.tau_huge + 1, s);
        TTC_CUDA(cudaMemcpyAsync(g->shard_eoff.get(), eo.data(), (nh + 1) * 8, cudaMemcpyHostToDevice, s));
        TTC_CUDA(cudaStreamSynchronize(s));  // eo is about to go out of scope
        const size_t bytes = heavy_scratch_bytes(g) * huge_pass_queries(g, k);
        if (g->scratch.count < bytes) g->scratch.alloc(bytes, s);
        b.huge = huge_args(g, g->scratch.get());
        b.huge_qcap = huge_pass_queries(g, k);
        b.huge.tri += lo[3];
        b.huge.eoff = g->shard_eoff.get();
        b.huge.nh = nh;
        b.huge.total = eo[nh];
    }
    count_bins(g, b, dq, k, acc, s);
}

void count_one_into(ttc_graph *g, const int64_t *dq, unsigned long long *acc, void *scratch, cudaStream_t s) {
    ProfOff off;  // no timing events: the caller's handle may be profiled by another thread
    count_graph(g, dq, 1, acc, scratch, s);
}

uint32_t fused_capacity(int wide) { return wide ? FusedCap<unsigned long long>::CAP : FusedCap<uint32_t>::CAP; }
uint32_t warp_capacity(int wide) { return wide ? WarpCap<unsigned long long>::CAP : WarpCap<uint32_t>::CAP; }

unsigned int take_bounds_word() {
#if TTC_DEBUG_BOUNDS
    unsigned int w = 0;
    const unsigned int zero = 0;
    TTC_CUDA(cudaMemcpyFromSymbol(&w, g_bounds_bad, sizeof w));
    TTC_CUDA(cudaMemcpyToSymbol(g_bounds_bad, &zero, sizeof zero));
    return w;
#else
    return 0;
#endif
}

// ---------------------------------------------------------------- per-triangle output
namespace {

// Per-triangle counts under dq of the triangles listed, in ascending order,
// in `all` (host ids into the graph's triangle list): d_out (device,
// zeroed, 8 per listed triangle in list order).  The ids fall in the bins
// in order (light, one-warp, one-CTA, flat), so each bin's share is one
// run of the list and its kernels write their rows in list order.
void count_ids(ttc_graph *g, const int64_t *dq, const std::vector<uint64_t> &all, unsigned long long *d_out,
               unsigned long long *flag, cudaStream_t s) {
    const uint64_t n = all.size();
    if (!n) return;
    const uint64_t nl = g->st.tau_light, nw = g->st.tau_hwarp, nc = g->st.tau_hcta;
    // d_idx: light ids, bin-relative heavy ids, absolute huge ids
    std::vector<uint64_t> order(n);
    uint64_t nlc = 0, nwc = 0, ncc = 0;
    for (uint64_t i = 0; i < n; i++) {
        const uint64_t ti = all[i];
        if (ti < nl) { order[i] = ti; nlc++; }
        else if (ti < nl + nw) { order[i] = ti - nl; nwc++; }
        else if (ti < nl + nw + nc) { order[i] = ti - nl - nw; ncc++; }
        else order[i] = ti;
    }
    const uint64_t nfc = nwc + ncc, nhc = n - nlc - nfc;
    DevBuf<uint64_t> d_idx(n, s);
    TTC_CUDA(cudaMemcpyAsync(d_idx.get(), order.data(), n * 8, cudaMemcpyHostToDevice, s));
    if (nlc) {
        if (g->strict)
            light_kernel<2, 1, true><<<light_grid((nlc + 31) / 32), LIGHT_THREADS, 0, s>>>(
                g->view.get(), g->prefix.get(), 1, dq, 1, d_out, flag, d_idx.get(), nlc);
        else
            light_kernel<2, 1, false><<<light_grid((nlc + 31) / 32), LIGHT_THREADS, 0, s>>>(
                g->view.get(), g->prefix.get(), 1, dq, 1, d_out, flag, d_idx.get(), nlc);
        TTC_LAUNCH_CHECK();
    }
    if (nwc)
        launch_warp_any<2>(heavy_kind(g->heavy_wide, g->strict), g->view.get(), g->prefix.get() + 2, 1, nwc, dq, 1,
                           d_out + 8 * nlc, flag, d_idx.get() + nlc, nwc, s);
    if (ncc)
        launch_fused_any<2>(heavy_kind(g->heavy_wide, g->strict, g->st.heavy_merge == TTC_HEAVY_MERGE), g->view.get(),
                            g->prefix.get() + 4, 1, ncc, dq, 1, d_out + 8 * (nlc + nwc), flag, d_idx.get() + nlc + nwc,
                            ncc, s);
    if (nhc) {
        DevBuf<uint4> sub(nhc, s);
        DevBuf<uint64_t> sizes(nhc, s), eoff(nhc + 1, s);
        record_sizes_kernel<<<ceil_div(nhc, 256), 256, 0, s>>>(g->tri.get(), d_idx.get() + nlc + nfc, nhc,
                                                               g->poff.get(), sub.get(), sizes.get());
        TTC_LAUNCH_CHECK();
        exclusive_scan_u64(sizes.get(), eoff.get(), nhc, s);
        uint64_t total = 0;
        TTC_CUDA(cudaMemcpyAsync(&total, eoff.get() + nhc, 8, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        HugeArgs ha{};
        ha.gv = g->view_host;
        ha.tri = sub.get();
        ha.eoff = eoff.get();
        ha.nh = nhc;
        ha.total = total;
        const size_t bytes = ((size_t)total + 4 * nhc) * 8 * (g->heavy_wide ? 8 : 4);
        DevBuf<uint8_t> pre(bytes, s);
        ha.pre = pre.get();
        ha.per_tri = d_out + 8 * (nlc + nfc);
        ProfOff off;
        if (g->heavy_wide) run_huge<unsigned long long>(g, ha, dq, nullptr, flag, s);
        else run_huge<uint32_t>(g, ha, dq, nullptr, flag, s);
    }
}

// Adds each listed triangle's count (all eight types; triangles c0 ..
// c0 + cnt - 1 of the list, their rows in out) to its three vertices and its
// three pairs; a sum past 2^64 sets the overflow flag.
__global__ void participation_kernel(const uint4 *tri, const uint2 *pv, uint64_t c0, uint64_t cnt,
                                     const unsigned long long *out, unsigned long long *vertex,
                                     unsigned long long *pair, unsigned long long *flag) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long tot = 0;
        bool ovf = false;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const unsigned long long x = out[8 * i + k];
            ovf |= tot + x < tot;
            tot += x;
        }
        if (!tot) continue;
        const uint4 r = tri[c0 + i];
        const uint2 a = pv[r.x], b = pv[r.y];
        const uint32_t u = (a.x == b.x || a.x == b.y) ? a.x : a.y;
        const uint32_t vtx[3] = {u, a.x == u ? a.y : a.x, b.x == u ? b.y : b.x};
        if (vertex)
#pragma unroll
            for (int k = 0; k < 3; k++) ovf |= atomicAdd(vertex + vtx[k], tot) + tot < tot;
        if (pair) {
            const uint32_t ps[3] = {r.x, r.y, r.z};
#pragma unroll
            for (int k = 0; k < 3; k++) ovf |= atomicAdd(pair + ps[k], tot) + tot < tot;
        }
        if (ovf) atomicOr(flag, 1ull);
    }
}

}  // namespace

void count_sample(ttc_graph *g, const int64_t *dq, uint64_t first, uint64_t stride, uint64_t cap,
                  uint32_t *tri_vtx_host, unsigned long long *out_host, uint64_t *written) {
    cudaStream_t s = g->stream;
    const uint64_t tau = g->st.tau;
    std::vector<uint64_t> all;
    for (uint64_t i = 0, ti = first; i < cap && ti < tau; i++, ti += stride) all.push_back(ti);
    *written = all.size();
    if (all.empty()) return;
    const uint64_t n = all.size();
    DevBuf<uint64_t> d_all(n, s);
    DevBuf<uint32_t> d_vtx(3 * n, s);
    DevBuf<unsigned long long> d_out(8 * n, s), flag(1, s);
    TTC_CUDA(cudaMemcpyAsync(d_all.get(), all.data(), n * 8, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemsetAsync(d_out.get(), 0, 8 * n * 8, s));
    TTC_CUDA(cudaMemsetAsync(flag.get(), 0, 8, s));
    record_vertices_kernel<<<ceil_div(n, 256), 256, 0, s>>>(g->tri.get(), g->pair_vtx.get(), d_all.get(), n,
                                                            d_vtx.get());
    TTC_LAUNCH_CHECK();
    count_ids(g, dq, all, d_out.get(), flag.get(), s);
    TTC_CUDA(cudaMemcpyAsync(out_host, d_out.get(), 8 * n * 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaMemcpyAsync(tri_vtx_host, d_vtx.get(), 3 * n * 4, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
}

void count_participation(ttc_graph *g, const int64_t *dq, uint64_t *vertex_host, uint64_t *pair_host) {
    cudaStream_t s = g->stream;
    const uint64_t tau = g->st.tau, n = g->st.n, ms = g->st.m_s;
    DevBuf<unsigned long long> vc(vertex_host ? (n ? n : 1) : 1, s), pc(pair_host ? (ms ? ms : 1) : 1, s), flag(1, s);
    if (vertex_host) TTC_CUDA(cudaMemsetAsync(vc.get(), 0, n * 8, s));
    if (pair_host) TTC_CUDA(cudaMemsetAsync(pc.get(), 0, ms * 8, s));
    TTC_CUDA(cudaMemsetAsync(flag.get(), 0, 8, s));
    // triangles in chunks, each counted per triangle and added to its
    // vertices and pairs
    const uint64_t chunk = uint64_t(1) << 22;
    DevBuf<unsigned long long> d_out(8 * std::min<uint64_t>(chunk, tau ? tau : 1), s);
    std::vector<uint64_t> ids;
    for (uint64_t c0 = 0; c0 < tau; c0 += chunk) {
        const uint64_t cnt = std::min(chunk, tau - c0);
        ids.resize(cnt);
        for (uint64_t i = 0; i < cnt; i++) ids[i] = c0 + i;
        TTC_CUDA(cudaMemsetAsync(d_out.get(), 0, 8 * cnt * 8, s));
        count_ids(g, dq, ids, d_out.get(), flag.get(), s);
        participation_kernel<<<ceil_div(cnt, 256), 256, 0, s>>>(g->tri.get(), g->pair_vtx.get(), c0, cnt,
                                                                d_out.get(), vertex_host ? vc.get() : nullptr,
                                                                pair_host ? pc.get() : nullptr, flag.get());
        TTC_LAUNCH_CHECK();
        TTC_CUDA(cudaStreamSynchronize(s));  // ids is rewritten for the next chunk
    }
    unsigned long long f = 0;
    TTC_CUDA(cudaMemcpyAsync(&f, flag.get(), 8, cudaMemcpyDeviceToHost, s));
    if (vertex_host && n) TTC_CUDA(cudaMemcpyAsync(vertex_host, vc.get(), n * 8, cudaMemcpyDeviceToHost, s));
    if (pair_host && ms) TTC_CUDA(cudaMemcpyAsync(pair_host, pc.get(), ms * 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    check_count_flag(f);
}

// ---------------------------------------------------------------- many graphs
void count_multi_launch(const MultiTable &t, const int64_t *dq, unsigned long long *acc, int light_per_sm,
                        int heavy_per_sm, cudaStream_t s) {
    unsigned long long *flag = acc + 8 * (size_t)t.G;
    if (t.chunks) {
        if (t.strict)
            light_kernel<0, 1, true><<<light_grid(t.chunks, light_per_sm), LIGHT_THREADS, 0, s>>>(
                t.gvs, t.chunk_pre, t.G, dq, 1, acc, flag, nullptr, 0);
        else
            light_kernel<0, 1, false><<<light_grid(t.chunks, light_per_sm), LIGHT_THREADS, 0, s>>>(
                t.gvs, t.chunk_pre, t.G, dq, 1, acc, flag, nullptr, 0);
        TTC_LAUNCH_CHECK();
    }
    for (int wide = 0; wide < 2; wide++) {
        if (!(wide ? t.any_wide : t.any_narrow)) continue;
        if (t.hwarp)
            launch_warp_any<0>(heavy_kind(wide, t.strict), t.gvs, t.hwarp_pre, t.G, t.hwarp, dq, 1, acc, flag, nullptr, 0, s,
                               2 * heavy_per_sm);
        if (t.hcta)
            launch_fused_any<0>(heavy_kind(wide, t.strict), t.gvs, t.hcta_pre, t.G, t.hcta, dq, 1, acc, flag, nullptr, 0, s, heavy_per_sm);
    }
}

void count_huge_of(ttc_graph *g, const int64_t *dq_one, unsigned long long *acc_row, unsigned long long *flag,
                   void *scratch, cudaStream_t s) {
    if (!g->st.tau_huge) return;
    const HugeArgs ha = huge_args(g, scratch);
    if (g->heavy_wide) run_huge<unsigned long long>(g, ha, dq_one, acc_row, flag, s);
    else run_huge<uint32_t>(g, ha, dq_one, acc_row, flag, s);
}

}  // namespace ttc
