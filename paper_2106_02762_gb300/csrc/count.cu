// Per-query counting (Alg. 1, counting step): for every static triangle
// <u, v, w> and every temporal ordering pi and orientation rho, the number of
// (d13, d12, d23)-temporal triangles, added to the type psi(pi, rho)
// (Table 1).  Only the edge lists of the pairs A = {u, v} and B = {u, w} are
// enumerated; the list of C = {v, w} is only searched (Sec. 5).
//
// Two bins, chosen per triangle at load time:
//
// light  (sigma_A * sigma_B small): one thread per triangle sums Lemma 1
//        directly over the pairs (a, b) in A x B.  With x the earlier and y
//        the later of a, b (key order), C's edge c can be
//          third  (x, y, c): t_y - t_x <= d12, key(c) > key(y),
//                            t_c <= min(t_y + d23, t_x + d13)      (Lemma 1)
//          second (x, c, y): t_y - t_x <= d13, key(x) < key(c) < key(y),
//                            t_c <= t_x + d12, t_c >= t_y - d23
//          first  (c, x, y): t_y - t_x <= d23, key(c) < key(x),
//                            t_c >= max(t_x - d12, t_y - d13)
//        and each case is a contiguous index range of C's key-sorted list.
//
// heavy  (prefix-sum form of Algs. 2-4, re-derived with key order for ties):
//        each enumerated edge e of A or B first gets, per direction of C,
//          h(e) = #{c: t_c <= t_e + d13}          (CEC_{+d13} terms, Alg. 2)
//          L(e) = #{c: key(c) < key(e)}           (CEC_{-inf} terms, Alg. 3)
//          R(e) = #{c: t_c <  t_e - d23}          (CEC_{-d23} terms, Alg. 3)
//          M(e) = #{c: t_c <  t_e - d13}          (CEC_{-d13} terms, Alg. 4)
//        whose prefix sums over each list (per own direction) are then read
//        at binary-searched range ends while enumerating the other list.  The
//        work is flat over all enumerated edges of all heavy triangles, so a
//        triangle with long lists is spread over many warps and CTAs.
//
// Deltas arrive normalised (d12, d23 <= d13 <= d12 + d23); all counts use
// unsigned 64-bit sums with carry detection.
#include <cstring>
#include <vector>

#include "graph.cuh"

namespace ttc {

namespace {

// Table 1: psi(pi_k, rho_r) = T_(value + 1); rows pi_1..pi_6, columns rho_1..rho_8.
__constant__ uint8_t PSI[6][8] = {
    {6, 5, 4, 7, 2, 1, 3, 0},
    {4, 2, 6, 3, 5, 0, 7, 1},
    {2, 1, 0, 3, 6, 5, 7, 4},
    {0, 6, 2, 7, 1, 4, 3, 5},
    {5, 0, 1, 7, 4, 2, 3, 6},
    {1, 4, 5, 3, 0, 6, 7, 2},
};
// Fig. 4: index of rho from the directions (dA, dB, dC) of the three pairs,
// code = 4 dA + 2 dB + dC, direction 0 being u->v, u->w, v->w.
//   rho_1 = (0,0,0), rho_2 = (0,1,1), rho_3 = (0,0,1), rho_4 = (0,1,0),
//   rho_5 = (1,0,0), rho_6 = (1,1,1), rho_7 = (1,0,1), rho_8 = (1,1,0)
__constant__ uint8_t RHO_OF_CODE[8] = {0, 2, 3, 1, 4, 6, 7, 5};

// Temporal orderings (Fig. 3), 0-based: pi_1 = A,B,C  pi_2 = B,A,C  pi_3 = A,C,B
// pi_4 = B,C,A  pi_5 = C,A,B  pi_6 = C,B,A  (first, second, third pair).
enum { PI1 = 0, PI2 = 1, PI3 = 2, PI4 = 3, PI5 = 4, PI6 = 5 };

__device__ __forceinline__ int type_of(int pi, uint32_t dA, uint32_t dB, uint32_t dC) {
    return PSI[pi][RHO_OF_CODE[(dA << 2) | (dB << 1) | dC]];
}

struct Query {
    int64_t d13, d12, d23;
};

__device__ __forceinline__ Query load_query(const int64_t *dq, uint32_t q) {
    return Query{dq[3 * q], dq[3 * q + 1], dq[3 * q + 2]};
}

// One pair's edge list: key[b .. b + n), plus the direction bookkeeping.
struct List {
    uint32_t b, n;
    uint32_t flip;  // 1: effective direction = stored direction ^ 1
};

struct KeyCtx {
    const int64_t *__restrict__ key;
    const uint32_t *__restrict__ fwd;
    int shift;
    int64_t span;
};

// number of elements of L with key < bound (bound >= 0)
__device__ __forceinline__ uint32_t count_below(const KeyCtx &k, const List &L, int64_t bound) {
    const int64_t *p = k.key + L.b;
    uint32_t lo = 0, n = L.n;
    while (n > 0) {
        const uint32_t half = n >> 1;
        if (__ldg(p + lo + half) < bound) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}
// #{e in L : key(e) < key(x)} for an edge x not in L
__device__ __forceinline__ uint32_t cnt_key(const KeyCtx &k, const List &L, int64_t kx) {
    return count_below(k, L, kx & ~int64_t(1));
}
// #{e in L : t(e) - t_min <= x}
__device__ __forceinline__ uint32_t cnt_le(const KeyCtx &k, const List &L, int64_t x) {
    if (x < 0) return 0;
    if (x >= k.span) return L.n;
    return count_below(k, L, (x + 1) << k.shift);
}
// #{e in L : t(e) - t_min < x}
__device__ __forceinline__ uint32_t cnt_lt(const KeyCtx &k, const List &L, int64_t x) { return cnt_le(k, L, x - 1); }
// number of direction-0 (effective) edges among the first `pos` of L
__device__ __forceinline__ uint32_t dir0(const KeyCtx &k, const List &L, uint32_t pos) {
    const uint32_t s0 = __ldg(k.fwd + L.b + pos) - __ldg(k.fwd + L.b);
    return L.flip ? pos - s0 : s0;
}

__device__ __forceinline__ List make_list(const uint32_t *__restrict__ poff, uint32_t p, uint32_t flip) {
    const uint32_t b = __ldg(poff + p);
    return List{b, __ldg(poff + p + 1) - b, flip};
}

// 64-bit accumulation with carry detection
__device__ __forceinline__ void add_checked(unsigned long long &acc, unsigned long long x, unsigned &ovf) {
    const unsigned long long r = acc + x;
    ovf |= r < acc;
    acc = r;
}

__device__ __forceinline__ void flush_block(unsigned long long (*s_acc)[256], int nthreads, unsigned long long *acc,
                                            unsigned ovf) {
    // s_acc[type][thread] -> global acc[type], one atomic per type per block
    __syncthreads();
    if (threadIdx.x < 8) {
        unsigned long long sum = 0;
        unsigned o = 0;
        for (int i = 0; i < nthreads; i++) add_checked(sum, s_acc[threadIdx.x][i], o);
        if (sum) {
            const unsigned long long old = atomicAdd(acc + threadIdx.x, sum);
            o |= old + sum < old;
        }
        if (o) atomicOr(reinterpret_cast<unsigned int *>(acc + 8), 1u);
    }
    if (ovf) atomicOr(reinterpret_cast<unsigned int *>(acc + 8), 1u);
}

// ---------------------------------------------------------------- light bin
constexpr int LIGHT_THREADS = 256;

struct LightArgs {
    KeyCtx k;
    const uint32_t *__restrict__ poff;
    const uint4 *__restrict__ tri;
    uint64_t ntri;
    // sample mode: triangle index = first + i * stride, counts to out[i][8]
    uint64_t first, stride;
    unsigned long long *per_tri;
};

// Adds the counts of one pair (x, y) of enumerated edges (x earlier) for all
// three positions of C's edge.  xa: x is on A (else on B).
template <typename Acc>
__device__ __forceinline__ void light_pair(const KeyCtx &k, const List &C, const Query &q, bool xa, int64_t rx,
                                           int64_t ry, uint32_t posCx, uint32_t posCy, uint32_t dA, uint32_t dB,
                                           Acc &&acc) {
    const int64_t gap = ry - rx;
    if (gap <= q.d12) {  // C third
        const int64_t lim = min(ry + q.d23, rx + q.d13);
        const uint32_t hi = cnt_le(k, C, lim), lo = posCy;
        if (hi > lo) {
            const uint32_t n0 = dir0(k, C, hi) - dir0(k, C, lo);
            const int pi = xa ? PI1 : PI2;
            acc(type_of(pi, dA, dB, 0), n0);
            acc(type_of(pi, dA, dB, 1), (hi - lo) - n0);
        }
    }
    if (gap <= q.d13) {  // C second
        const uint32_t lo = max(posCx, cnt_lt(k, C, ry - q.d23));
        const uint32_t hi = min(posCy, cnt_le(k, C, rx + q.d12));
        if (hi > lo) {
            const uint32_t n0 = dir0(k, C, hi) - dir0(k, C, lo);
            const int pi = xa ? PI3 : PI4;
            acc(type_of(pi, dA, dB, 0), n0);
            acc(type_of(pi, dA, dB, 1), (hi - lo) - n0);
        }
    }
    if (gap <= q.d23) {  // C first
        const uint32_t lo = cnt_lt(k, C, max(rx - q.d12, ry - q.d13)), hi = posCx;
        if (hi > lo) {
            const uint32_t n0 = dir0(k, C, hi) - dir0(k, C, lo);
            const int pi = xa ? PI5 : PI6;
            acc(type_of(pi, dA, dB, 0), n0);
            acc(type_of(pi, dA, dB, 1), (hi - lo) - n0);
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-cooperative light kernel.  Each warp takes 32 consecutive triangle
// records, flattens their A x B pairs (fewer than light_max_pairs each) into
// one index space and gives every lane one pair per step, so lanes stay busy
// whatever the per-triangle list sizes.  Per pair: the two keys, their
// positions in C, and the three cases of light_pair.
constexpr int LIGHT_WARPS = LIGHT_THREADS / 32;

struct WarpTris {
    uint32_t excl[LIGHT_WARPS][33];  // exclusive prefix of pair counts
    uint4 lst[LIGHT_WARPS][32];      // A.b, B.b, C.b, C.n
    uint32_t bn[LIGHT_WARPS][32];    // B.n
    uint32_t fl[LIGHT_WARPS][32];    // flip flags
};

// MODE 0: one query, per-thread accumulators.  MODE 1: nq queries, block
// accumulators.  MODE 2: one query, per-triangle output for the sampled
// triangles idx[0 .. ntri) (acc is then [ntri][8]).
template <int MODE>
__global__ void __launch_bounds__(LIGHT_THREADS)
    light_kernel_warp(LightArgs a, const int64_t *dq, uint32_t nq, unsigned long long *acc, const uint64_t *idx) {
    __shared__ WarpTris wt;
    __shared__ unsigned long long s_acc[MODE == 0 ? 8 : 1][MODE == 0 ? 256 : 1];
    extern __shared__ unsigned long long s_bacc[];  // MODE 1: [nq * 8]
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
    }
    if (MODE == 1) {
        for (uint32_t i = threadIdx.x; i < nq * 8; i += blockDim.x) s_bacc[i] = 0;
        __syncthreads();
    }
    unsigned ovf = 0;
    const KeyCtx &k = a.k;
    const uint64_t nchunks = (a.ntri + 31) / 32;
    const uint64_t gw = (uint64_t)blockIdx.x * LIGHT_WARPS + w, nw = (uint64_t)gridDim.x * LIGHT_WARPS;
    const Query Q0 = load_query(dq, 0);
    int64_t gmax = Q0.d13;  // every case needs t_y - t_x <= d13 (normalised)
    if (MODE == 1)
        for (uint32_t q = 1; q < nq; q++) gmax = max(gmax, dq[3 * q]);
    for (uint64_t c = gw; c < nchunks; c += nw) {
        const uint64_t ti = c * 32 + lane;
        uint32_t npairs = 0;
        if (ti < a.ntri) {
            const uint4 r = __ldg(a.tri + (MODE == 2 ? idx[ti] : ti));
            const uint32_t ab = __ldg(a.poff + r.x), an = __ldg(a.poff + r.x + 1) - ab;
            const uint32_t bb = __ldg(a.poff + r.y), bn = __ldg(a.poff + r.y + 1) - bb;
            const uint32_t cb = __ldg(a.poff + r.z), cn = __ldg(a.poff + r.z + 1) - cb;
            npairs = an * bn;
            wt.lst[w][lane] = make_uint4(ab, bb, cb, cn);
            wt.bn[w][lane] = bn;
            wt.fl[w][lane] = r.w;
        }
        uint32_t x = npairs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        wt.excl[w][lane] = x - npairs;
        const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
        if (lane == 0) wt.excl[w][32] = total;
        __syncwarp();
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t j = base + lane;
            if (j >= total) continue;
            uint32_t o = 0;  // last slot with excl <= j (skips empty slots before it)
#pragma unroll
            for (uint32_t step = 16; step; step >>= 1)
                if (wt.excl[w][o + step] <= j) o += step;
            const uint4 L = wt.lst[w][o];
            const uint32_t bn = wt.bn[w][o], fl = wt.fl[w][o];
            const uint32_t loc = j - wt.excl[w][o];
            const uint32_t ai = loc / bn, bi = loc - ai * bn;
            const int64_t ka = __ldg(k.key + L.x + ai), kb = __ldg(k.key + L.y + bi);
            const int64_t ra = ka >> k.shift, rb = kb >> k.shift;
            const bool a_first = ka < kb;
            const int64_t gap = a_first ? rb - ra : ra - rb;
            if (gap > gmax) continue;
            const List C{L.z, L.w, (fl & TriRec::FLIP_C) ? 1u : 0u};
            const uint32_t dA = (uint32_t)(ka & 1) ^ (fl & TriRec::FLIP_A);
            const uint32_t dB = (uint32_t)(kb & 1) ^ ((fl & TriRec::FLIP_B) ? 1u : 0u);
            const uint32_t pa = cnt_key(k, C, ka), pb = cnt_key(k, C, kb);
            for (uint32_t q = 0; q < (MODE == 1 ? nq : 1u); q++) {
                const Query Q = MODE == 1 ? load_query(dq, q) : Q0;
                auto accq = [&](int type, uint32_t n) {
                    if constexpr (MODE == 0) add_checked(s_acc[type][threadIdx.x], n, ovf);
                    else if constexpr (MODE == 1) atomicAdd(&s_bacc[q * 8 + type], (unsigned long long)n);
                    else atomicAdd(acc + 8 * (c * 32 + o) + type, (unsigned long long)n);
                };
                if (a_first) light_pair(k, C, Q, true, ra, rb, pa, pb, dA, dB, accq);
                else light_pair(k, C, Q, false, rb, ra, pb, pa, dA, dB, accq);
            }
        }
        __syncwarp();
    }
    if constexpr (MODE == 0) flush_block(s_acc, LIGHT_THREADS, acc, ovf);
    if constexpr (MODE == 1) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nq * 8; i += blockDim.x)
            if (s_bacc[i]) atomicAdd(acc + i, s_bacc[i]);
    }
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

__global__ void gather_records_kernel(const uint4 *tri, const uint64_t *idx, uint64_t count, const uint32_t *poff,
                                      uint4 *out, uint64_t *sizes) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = tri[idx[i]];
        out[i] = r;
        sizes[i] = (poff[r.x + 1] - poff[r.x]) + (poff[r.y + 1] - poff[r.y]);
    }
}

// ---------------------------------------------------------------- heavy bin
constexpr int HEAVY_THREADS = 256;

struct HeavyArgs {
    KeyCtx k;
    const uint32_t *__restrict__ poff;
    const uint4 *__restrict__ tri;      // heavy records
    const uint64_t *__restrict__ eoff;  // [nh + 1]
    uint64_t nh, total;
    void *pre;                          // prefix entries: 8 values each
    // sample mode: per-record output slots (nullptr otherwise)
    unsigned long long *per_tri;
};

// Locates enumerated element g: its triangle h and index j in A ++ B.
__device__ __forceinline__ uint64_t find_tri(const uint64_t *__restrict__ eoff, uint64_t nh, uint64_t g) {
    uint64_t lo = 0, hi = nh;  // last h with eoff[h] <= g
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldg(eoff + mid) <= g) lo = mid; else hi = mid;
    }
    return lo;
}

struct HeavyTri {
    List A, B, C;
    uint32_t a0, b0;  // effective direction-0 counts of A and B
    uint64_t base;    // first prefix entry of this triangle
};

__device__ __forceinline__ HeavyTri heavy_tri(const HeavyArgs &a, uint64_t h) {
    const uint4 r = __ldg(a.tri + h);
    HeavyTri t;
    t.A = make_list(a.poff, r.x, r.w & TriRec::FLIP_A);
    t.B = make_list(a.poff, r.y, (r.w & TriRec::FLIP_B) ? 1u : 0u);
    t.C = make_list(a.poff, r.z, (r.w & TriRec::FLIP_C) ? 1u : 0u);
    t.a0 = dir0(a.k, t.A, t.A.n);
    t.b0 = dir0(a.k, t.B, t.B.n);
    t.base = __ldg(a.eoff + h) + 4 * h;
    return t;
}

// first prefix entry of the own-direction-d segment of list Z (0 = A, 1 = B)
__device__ __forceinline__ uint64_t seg_base(const HeavyTri &t, int z, uint32_t d) {
    uint64_t b = t.base;
    if (z) b += t.A.n + 2;
    const uint32_t n0 = z ? t.b0 : t.a0;
    if (d) b += n0 + 1;
    return b;
}

template <typename P>
__global__ void __launch_bounds__(HEAVY_THREADS) heavy_phase1(HeavyArgs a, const int64_t *dq) {
    const Query q = load_query(dq, 0);
    P *pre = static_cast<P *>(a.pre);
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t h = find_tri(a.eoff, a.nh, g);
        const HeavyTri t = heavy_tri(a, h);
        uint32_t j = (uint32_t)(g - __ldg(a.eoff + h));
        const int z = j >= t.A.n;
        const List &Z = z ? t.B : t.A;
        if (z) j -= t.A.n;
        const int64_t ke = __ldg(a.k.key + Z.b + j);
        const int64_t re = ke >> a.k.shift;
        const uint32_t d = (uint32_t)(ke & 1) ^ Z.flip;
        const uint32_t z0 = dir0(a.k, Z, j);
        const uint32_t rank = d ? j - z0 : z0;
        const uint32_t ph = cnt_le(a.k, t.C, re + q.d13);
        const uint32_t pl = cnt_key(a.k, t.C, ke);
        const uint32_t pr = cnt_lt(a.k, t.C, re - q.d23);
        const uint32_t pm = cnt_lt(a.k, t.C, re - q.d13);
        const uint32_t h0 = dir0(a.k, t.C, ph), l0 = dir0(a.k, t.C, pl), r0 = dir0(a.k, t.C, pr),
                       m0 = dir0(a.k, t.C, pm);
        P *e = pre + 8 * (seg_base(t, z, d) + rank + 1);
        e[0] = h0; e[1] = ph - h0;
        e[2] = l0; e[3] = pl - l0;
        e[4] = r0; e[5] = pr - r0;
        e[6] = m0; e[7] = pm - m0;
    }
}

// Inclusive scan of each own-direction segment (entry 0 of a segment is 0).
// One warp per segment; 4 segments per heavy triangle.
template <typename P>
__global__ void __launch_bounds__(HEAVY_THREADS) heavy_scan(HeavyArgs a) {
    P *pre = static_cast<P *>(a.pre);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t sidx = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sidx < 4 * a.nh;
         sidx += warps) {
        const uint64_t h = sidx >> 2;
        const int z = (int)((sidx >> 1) & 1);
        const uint32_t d = (uint32_t)(sidx & 1);
        const HeavyTri t = heavy_tri(a, h);
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

// Prefix of slot s over the own-direction-d segment of Z, first `cnt` entries.
template <typename P>
__device__ __forceinline__ unsigned long long pref(const P *pre, uint64_t sb, uint32_t cnt, int s) {
    return (unsigned long long)pre[8 * (sb + cnt) + s];
}

template <typename P>
__global__ void __launch_bounds__(HEAVY_THREADS) heavy_phase2(HeavyArgs a, const int64_t *dq, unsigned long long *acc) {
    __shared__ unsigned long long s_acc[8][256];
#pragma unroll
    for (int j = 0; j < 8; j++) s_acc[j][threadIdx.x] = 0;
    unsigned ovf = 0;
    const Query q = load_query(dq, 0);
    const P *pre = static_cast<const P *>(a.pre);
    const KeyCtx &k = a.k;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t h = find_tri(a.eoff, a.nh, g);
        const HeavyTri t = heavy_tri(a, h);
        uint32_t j = (uint32_t)(g - __ldg(a.eoff + h));
        const int z = j >= t.A.n;  // this edge's list Z (0 = A, 1 = B); O is the other
        if (z) j -= t.A.n;
        const List &Z = z ? t.B : t.A;
        const List &O = z ? t.A : t.B;
        const int oz = 1 - z;
        const int64_t ke = __ldg(k.key + Z.b + j);
        const int64_t re = ke >> k.shift;
        const uint32_t de = (uint32_t)(ke & 1) ^ Z.flip;
        unsigned long long *pt = a.per_tri ? a.per_tri + 8 * h : nullptr;
        auto add = [&](uint32_t dO, uint32_t dC, int pi_if_z_is_a, int pi_if_z_is_b, unsigned long long n) {
            if (!n) return;
            const uint32_t dA = z ? dO : de, dB = z ? de : dO;
            const int type = type_of(z ? pi_if_z_is_b : pi_if_z_is_a, dA, dB, dC);
            if (pt) atomicAdd(pt + type, n);
            else add_checked(s_acc[type][threadIdx.x], n, ovf);
        };
        // searches in C (split by C's direction)
        const uint32_t posC = cnt_key(k, t.C, ke);
        const uint32_t K0 = dir0(k, t.C, posC), K1 = posC - K0;
        const uint32_t pH = cnt_le(k, t.C, re + q.d23);
        const uint32_t H0 = dir0(k, t.C, pH), H1 = pH - H0;
        const uint32_t pG = cnt_le(k, t.C, re + q.d12);
        const uint32_t G0 = dir0(k, t.C, pG), G1 = pG - G0;
        const uint32_t pLo = cnt_lt(k, t.C, re - q.d12);
        const uint32_t Lo0 = dir0(k, t.C, pLo), Lo1 = pLo - Lo0;
        const uint32_t Kd[2] = {K0, K1}, Hd[2] = {H0, H1}, Gd[2] = {G0, G1}, Lod[2] = {Lo0, Lo1};
        // searches in O (merged positions)
        const uint32_t posO = cnt_key(k, O, ke);
        const uint32_t o_lo = min(cnt_lt(k, O, re - q.d12), posO);
        const uint32_t o_mid = min(max(cnt_le(k, O, re + q.d23 - q.d13), o_lo), posO);
        const uint32_t r1 = max(cnt_le(k, O, re + min(q.d12, q.d23)), posO);
        const uint32_t r2 = max(cnt_le(k, O, re + max(q.d12, q.d23)), r1);
        const uint32_t r3 = max(cnt_le(k, O, re + q.d13), r2);
        const uint32_t sp = max(cnt_le(k, O, re + q.d13 - q.d12), posO);
        const uint32_t en = max(cnt_le(k, O, re + q.d23), sp);
        const uint32_t pos[9] = {o_lo, o_mid, posO, r1, r2, r3, sp, en, 0};
        for (uint32_t dO = 0; dO < 2; dO++) {
            // own-direction-dO ranks of the merged positions in O
            uint32_t c[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const uint32_t d0 = dir0(k, O, pos[i]);
                c[i] = dO ? pos[i] - d0 : d0;
            }
            const uint32_t c_lo = c[0], c_mid = c[1], c_pos = c[2], c_r1 = c[3], c_r2 = c[4], c_r3 = c[5],
                           c_sp = c[6], c_en = c[7];
            const uint64_t sb = seg_base(t, oz, dO);
            for (uint32_t dC = 0; dC < 2; dC++) {
                // (1) e second, O's edge first, C third: Alg. 2 (pi_1 / pi_2)
                {
                    const unsigned long long hsum = pref(pre, sb, c_mid, 0 + dC) - pref(pre, sb, c_lo, 0 + dC);
                    const unsigned long long n = hsum + (unsigned long long)Hd[dC] * (c_pos - c_mid) -
                                                 (unsigned long long)Kd[dC] * (c_pos - c_lo);
                    add(dO, dC, PI2, PI1, n);
                }
                // (2) e first, C second, O's edge third: Alg. 3 (pi_3 / pi_4)
                {
                    const unsigned long long L_1 = pref(pre, sb, c_r1, 2 + dC) - pref(pre, sb, c_pos, 2 + dC);
                    unsigned long long n = L_1 - (unsigned long long)Kd[dC] * (c_r1 - c_pos);
                    if (q.d12 <= q.d23) {
                        n += (unsigned long long)(Gd[dC] - Kd[dC]) * (c_r2 - c_r1);
                    } else {
                        n += (pref(pre, sb, c_r2, 2 + dC) - pref(pre, sb, c_r1, 2 + dC)) -
                             (pref(pre, sb, c_r2, 4 + dC) - pref(pre, sb, c_r1, 4 + dC));
                    }
                    n += (unsigned long long)Gd[dC] * (c_r3 - c_r2) -
                         (pref(pre, sb, c_r3, 4 + dC) - pref(pre, sb, c_r2, 4 + dC));
                    add(dO, dC, PI3, PI4, n);
                }
                // (3) C first, e second, O's edge third: Alg. 4 (pi_5 / pi_6)
                {
                    unsigned long long n = (unsigned long long)(Kd[dC] - Lod[dC]) * (c_sp - c_pos);
                    n += (unsigned long long)Kd[dC] * (c_en - c_sp) -
                         (pref(pre, sb, c_en, 6 + dC) - pref(pre, sb, c_sp, 6 + dC));
                    add(dO, dC, PI5, PI6, n);
                }
            }
        }
    }
    if (!a.per_tri) flush_block(s_acc, HEAVY_THREADS, acc, ovf);
}

template <typename P>
void run_heavy(ttc_graph *g, const HeavyArgs &ha, const int64_t *dq_one, unsigned long long *acc, cudaStream_t s) {
    const unsigned grid = (unsigned)(sm_count() * 8);
    prof_begin(g, s, "heavy_phase1");
    heavy_phase1<P><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
    prof_begin(g, s, "heavy_scan");
    heavy_scan<P><<<grid, HEAVY_THREADS, 0, s>>>(ha);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
    prof_begin(g, s, "heavy_phase2");
    heavy_phase2<P><<<grid, HEAVY_THREADS, 0, s>>>(ha, dq_one, acc);
    TTC_LAUNCH_CHECK();
    prof_end(g, s);
}

HeavyArgs heavy_args(ttc_graph *g, cudaStream_t s) {
    HeavyArgs ha{};
    ha.k = KeyCtx{g->key.get(), g->fwd.get(), g->shift, g->span};
    ha.poff = g->poff.get();
    ha.tri = g->tri.get() + g->st.tau_light;
    ha.eoff = g->heavy_eoff.get();
    ha.nh = g->st.tau_heavy;
    ha.total = g->heavy_elems;
    const size_t entries = (size_t)g->heavy_elems + 4 * (size_t)g->st.tau_heavy;
    const size_t bytes = entries * 8 * (g->heavy_wide ? 8 : 4);
    if (g->scratch.count < bytes) g->scratch.alloc(bytes, s);
    ha.pre = g->scratch.get();
    return ha;
}

constexpr int MAX_BATCH_SMEM_Q = 256;

unsigned light_grid(uint64_t ntri) {
    const uint64_t want = (ntri + LIGHT_THREADS - 1) / LIGHT_THREADS;
    const uint64_t cap = (uint64_t)sm_count() * 8;
    return (unsigned)(want < 1 ? 1 : want < cap ? want : cap);
}

LightArgs light_args(ttc_graph *g) {
    LightArgs la{};
    la.k = KeyCtx{g->key.get(), g->fwd.get(), g->shift, g->span};
    la.poff = g->poff.get();
    la.tri = g->tri.get();
    la.ntri = g->st.tau_light;
    return la;
}

}  // namespace

void count_queue(ttc_graph *g, const int64_t *dq, uint32_t k, unsigned long long *acc, cudaStream_t s) {
    if (!g->st.tau || !k) return;
    const LightArgs la = light_args(g);
    if (la.ntri) {
        const unsigned grid = light_grid(la.ntri);
        if (k == 1) {
            prof_begin(g, s, "light");
            light_kernel_warp<0><<<grid, LIGHT_THREADS, 0, s>>>(la, dq, 1, acc, nullptr);
            TTC_LAUNCH_CHECK();
            prof_end(g, s);
        } else {
            for (uint32_t q0 = 0; q0 < k; q0 += MAX_BATCH_SMEM_Q) {
                const uint32_t nq = k - q0 < (uint32_t)MAX_BATCH_SMEM_Q ? k - q0 : (uint32_t)MAX_BATCH_SMEM_Q;
                prof_begin(g, s, "light_batch");
                light_kernel_warp<1><<<grid, LIGHT_THREADS, nq * 8 * sizeof(unsigned long long), s>>>(
                    la, dq + 3 * (size_t)q0, nq, acc + 8 * (size_t)q0, nullptr);
                TTC_LAUNCH_CHECK();
                prof_end(g, s);
            }
        }
    }
    if (g->st.tau_heavy) {
        const HeavyArgs ha = heavy_args(g, s);
        for (uint32_t q = 0; q < k; q++) {
            if (g->heavy_wide) run_heavy<unsigned long long>(g, ha, dq + 3 * q, acc + 8 * (size_t)q, s);
            else run_heavy<uint32_t>(g, ha, dq + 3 * q, acc + 8 * (size_t)q, s);
        }
    }
}

size_t heavy_scratch_bytes(const ttc_graph *g) {
    const size_t entries = (size_t)g->heavy_elems + 4 * (size_t)g->st.tau_heavy;
    return g->st.tau_heavy ? entries * 8 * (g->heavy_wide ? 8 : 4) : 0;
}

void count_one_into(ttc_graph *g, const int64_t *dq, unsigned long long *acc, void *scratch, cudaStream_t s) {
    if (!g->st.tau) return;
    const LightArgs la = light_args(g);
    if (la.ntri) {
        light_kernel_warp<0><<<light_grid(la.ntri), LIGHT_THREADS, 0, s>>>(la, dq, 1, acc, nullptr);
        TTC_LAUNCH_CHECK();
    }
    if (g->st.tau_heavy) {
        HeavyArgs ha{};
        ha.k = KeyCtx{g->key.get(), g->fwd.get(), g->shift, g->span};
        ha.poff = g->poff.get();
        ha.tri = g->tri.get() + g->st.tau_light;
        ha.eoff = g->heavy_eoff.get();
        ha.nh = g->st.tau_heavy;
        ha.total = g->heavy_elems;
        ha.pre = scratch;
        const bool saved = g->profiling;
        g->profiling = false;
        if (g->heavy_wide) run_heavy<unsigned long long>(g, ha, dq, acc, s);
        else run_heavy<uint32_t>(g, ha, dq, acc, s);
        g->profiling = saved;
    }
}

void count_sample(ttc_graph *g, const int64_t *dq, uint64_t first, uint64_t stride, uint64_t cap,
                  uint32_t *tri_vtx_host, unsigned long long *out_host, uint64_t *written) {
    cudaStream_t s = g->stream;
    const uint64_t tau = g->st.tau, nl = g->st.tau_light;
    std::vector<uint64_t> li, hi_, all;
    for (uint64_t i = 0, ti = first; i < cap && ti < tau; i++, ti += stride) {
        all.push_back(ti);
        (ti < nl ? li : hi_).push_back(ti);
    }
    *written = all.size();
    if (all.empty()) return;
    const uint64_t n = all.size(), nlc = li.size(), nhc = hi_.size();
    DevBuf<uint64_t> d_all(n, s), d_idx(n, s);
    DevBuf<uint32_t> d_vtx(3 * n, s);
    DevBuf<unsigned long long> d_out(8 * n, s);
    TTC_CUDA(cudaMemcpyAsync(d_all.get(), all.data(), n * 8, cudaMemcpyHostToDevice, s));
    TTC_CUDA(cudaMemsetAsync(d_out.get(), 0, 8 * n * 8, s));
    record_vertices_kernel<<<ceil_div(n, 256), 256, 0, s>>>(g->tri.get(), g->pair_vtx.get(), d_all.get(), n,
                                                            d_vtx.get());
    TTC_LAUNCH_CHECK();
    // light samples first, then heavy ones, in d_idx / d_out order
    std::vector<uint64_t> order(li);
    order.insert(order.end(), hi_.begin(), hi_.end());
    TTC_CUDA(cudaMemcpyAsync(d_idx.get(), order.data(), n * 8, cudaMemcpyHostToDevice, s));
    if (nlc) {
        LightArgs la = light_args(g);
        la.ntri = nlc;
        light_kernel_warp<2><<<light_grid(nlc), LIGHT_THREADS, 0, s>>>(la, dq, 1, d_out.get(), d_idx.get());
        TTC_LAUNCH_CHECK();
    }
    if (nhc) {
        DevBuf<uint4> sub(nhc, s);
        DevBuf<uint64_t> sizes(nhc, s), eoff(nhc + 1, s);
        gather_records_kernel<<<ceil_div(nhc, 256), 256, 0, s>>>(g->tri.get(), d_idx.get() + nlc, nhc,
                                                                 g->poff.get(), sub.get(), sizes.get());
        TTC_LAUNCH_CHECK();
        exclusive_scan_u64(sizes.get(), eoff.get(), nhc, s);
        uint64_t total = 0;
        TTC_CUDA(cudaMemcpyAsync(&total, eoff.get() + nhc, 8, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        HeavyArgs ha{};
        ha.k = KeyCtx{g->key.get(), g->fwd.get(), g->shift, g->span};
        ha.poff = g->poff.get();
        ha.tri = sub.get();
        ha.eoff = eoff.get();
        ha.nh = nhc;
        ha.total = total;
        const size_t bytes = ((size_t)total + 4 * nhc) * 8 * (g->heavy_wide ? 8 : 4);
        DevBuf<uint8_t> pre(bytes, s);
        ha.pre = pre.get();
        ha.per_tri = d_out.get() + 8 * nlc;
        const bool saved = g->profiling;
        g->profiling = false;
        if (g->heavy_wide) run_heavy<unsigned long long>(g, ha, dq, nullptr, s);
        else run_heavy<uint32_t>(g, ha, dq, nullptr, s);
        g->profiling = saved;
    }
    std::vector<unsigned long long> h(8 * n);
    std::vector<uint32_t> hv(3 * n);
    TTC_CUDA(cudaMemcpyAsync(h.data(), d_out.get(), 8 * n * 8, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaMemcpyAsync(hv.data(), d_vtx.get(), 3 * n * 4, cudaMemcpyDeviceToHost, s));
    TTC_CUDA(cudaStreamSynchronize(s));
    // back to sample order
    for (uint64_t i = 0, a = 0, b = 0; i < n; i++) {
        const uint64_t slot = all[i] < nl ? a++ : nlc + b++;
        memcpy(out_host + 8 * i, &h[8 * slot], 64);
    }
    memcpy(tri_vtx_host, hv.data(), 3 * n * 4);
}

}  // namespace ttc
