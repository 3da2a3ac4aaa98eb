// Device-wide building blocks used by the load path: exclusive scans, a
// stable LSD radix sort and a min/max reduction.  All are plain CUDA written
// for this library (no CUB/Thrust).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "sort.cuh"

namespace ttc {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T *total) {
    // v: this thread's value; returns the sum over lower threads.
    __shared__ T warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    const T warp_off = warp ? warp_sums[warp - 1] : T(0);
    if (total) *total = warp_sums[SCAN_THREADS / 32 - 1];
    const T excl = warp_off + x - v;
    __syncthreads();  // warp_sums reused by the next call
    return excl;
}

template <typename T, typename In>
__global__ void __launch_bounds__(SCAN_THREADS) tile_sums_kernel(const In *in, size_t n, T *sums) {
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const size_t idx = base + (size_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += (T)in[idx];
    }
    T total;
    block_exclusive_scan<T>(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// SCAN_ITEMS consecutive items of one thread as whole 16-byte (or 8-byte)
// words, for tiles that lie wholly inside the array.
template <typename X>
__device__ __forceinline__ void load_items(const X *p, X (&v)[SCAN_ITEMS]) {
    constexpr int B = (int)sizeof(X) * SCAN_ITEMS;
    static_assert(B % 8 == 0, "item group of whole 8-byte words");
    if constexpr (B % 16 == 0) {
        uint4 w[B / 16];
#pragma unroll
        for (int i = 0; i < B / 16; i++) w[i] = reinterpret_cast<const uint4 *>(p)[i];
        memcpy(v, w, B);
    } else {
        uint2 w[B / 8];
#pragma unroll
        for (int i = 0; i < B / 8; i++) w[i] = reinterpret_cast<const uint2 *>(p)[i];
        memcpy(v, w, B);
    }
}
template <typename X>
__device__ __forceinline__ void store_items(X *p, const X (&v)[SCAN_ITEMS]) {
    constexpr int B = (int)sizeof(X) * SCAN_ITEMS;
    static_assert(B % 16 == 0, "item group of whole 16-byte words");
    uint4 w[B / 16];
    memcpy(w, v, B);
#pragma unroll
    for (int i = 0; i < B / 16; i++) reinterpret_cast<uint4 *>(p)[i] = w[i];
}

// VEC: in and out are aligned to a thread's item group (SCAN_ITEMS items),
// so full tiles move as whole words.
template <typename T, typename In, bool VEC>
__global__ void __launch_bounds__(SCAN_THREADS)
    tile_scan_kernel(const In *in, T *out, size_t n, const T *tile_off) {
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    const bool full = VEC && (size_t)(blockIdx.x + 1) * SCAN_TILE <= n;  // block-uniform
    T v[SCAN_ITEMS];
    T s = 0;
    if (full) {
        In x[SCAN_ITEMS];
        load_items<In>(in + base, x);
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            v[i] = (T)x[i];
            s += v[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            const size_t idx = base + i;
            v[i] = idx < n ? (T)in[idx] : T(0);
            s += v[i];
        }
    }
    T total;
    T run = block_exclusive_scan<T>(s, &total) + (tile_off ? tile_off[blockIdx.x] : T(0));
    if (full) {
        T o[SCAN_ITEMS];
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            o[i] = run;
            run += v[i];
        }
        store_items<T>(out + base, o);
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            const size_t idx = base + i;
            if (idx < n) out[idx] = run;
            run += v[i];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

template <typename T, typename In>
void exclusive_scan_impl(const In *in, T *out, size_t n, cudaStream_t s) {
    const unsigned tiles = n ? ceil_div(n, SCAN_TILE) : 1;
    if (tiles == 1) {
        tile_scan_kernel<T, In, false><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        TTC_LAUNCH_CHECK();
        return;
    }
    DevBuf<T> sums(tiles, s), offs(tiles + 1, s);
    tile_sums_kernel<T, In><<<tiles, SCAN_THREADS, 0, s>>>(in, n, sums.get());
    TTC_LAUNCH_CHECK();
    exclusive_scan_impl<T, T>(sums.get(), offs.get(), tiles, s);
    const bool vec = reinterpret_cast<uintptr_t>(in) % (sizeof(In) * SCAN_ITEMS) == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 16 == 0 && (sizeof(T) * SCAN_ITEMS) % 16 == 0;
    if (vec) tile_scan_kernel<T, In, true><<<tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs.get());
    else tile_scan_kernel<T, In, false><<<tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs.get());
    TTC_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;                         // per lane
constexpr int RS_WARP_TILE = 32 * RS_ITEMS;         // consecutive elements per warp
constexpr int RS_TILE = RS_WARPS * RS_WARP_TILE;    // elements per block
constexpr int RADIX_BITS = 8;                       // digit width (the last pass may use fewer)
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_DPT = RADIX / RS_THREADS;          // digits per thread in the per-digit steps

__global__ void __launch_bounds__(RS_THREADS)
    radix_hist_kernel(const uint64_t *keys, size_t n, int shift, uint32_t mask, uint32_t *counts, unsigned tiles) {
    __shared__ uint32_t hist[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) hist[d] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_TILE / RS_THREADS; i++) {
        const size_t idx = base + (size_t)i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&hist[(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    // digit-major layout: a flat exclusive scan gives each (digit, tile) its
    // output offset in stable order
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) counts[(size_t)d * tiles + blockIdx.x] = hist[d];
}

// Stable scatter of one digit.  Ranks come from warp-level match masks in
// element order; the tile is first reordered by digit in shared memory, then
// written out so that each digit's run is contiguous in global memory
// (coalesced stores).
template <typename V>
__global__ void __launch_bounds__(RS_THREADS)
    radix_scatter_kernel(const uint64_t *keys_in, const V *vals_in, uint64_t *keys_out, V *vals_out,
                         size_t n, int shift, uint32_t mask, const uint32_t *offsets, unsigned tiles) {
    __shared__ uint16_t wcnt[RS_WARPS][RADIX];  // per warp and digit (at most RS_WARP_TILE)
    __shared__ uint32_t dstart[RADIX];   // block-local start of each digit
    __shared__ uint32_t gstart[RADIX];   // global start of each digit for this tile
    extern __shared__ __align__(16) unsigned char rs_dyn[];
    uint64_t *s_key = reinterpret_cast<uint64_t *>(rs_dyn);
    V *s_val = reinterpret_cast<V *>(s_key + RS_TILE);
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const size_t tile_base = (size_t)blockIdx.x * RS_TILE;
    const size_t base = tile_base + (size_t)warp * RS_WARP_TILE;
    uint64_t k[RS_ITEMS];
    V v[RS_ITEMS];
    uint32_t local[RS_ITEMS];
    int dig[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        const size_t idx = base + (size_t)i * 32 + lane;
        const bool ok = idx < n;
        k[i] = ok ? keys_in[idx] : 0;
        v[i] = ok ? vals_in[idx] : V(0);
        dig[i] = ok ? (int)((k[i] >> shift) & mask) : RADIX;  // RADIX = padding
        const unsigned peers = __match_any_sync(0xffffffffu, dig[i]);
        const int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (ok) b = wcnt[warp][dig[i]];
        __syncwarp();
        if (ok && lane == leader) wcnt[warp][dig[i]] = (uint16_t)(b + __popc(peers));
        __syncwarp();
        local[i] = b + __popc(peers & lt_mask);
    }
    __syncthreads();
    {  // per digit: exclusive prefix over warps, the digit's block total, and
       // an exclusive scan of the totals (RS_DPT consecutive digits a thread)
        uint32_t tot[RS_DPT], sum = 0;
#pragma unroll
        for (int j = 0; j < RS_DPT; j++) {
            const int d = threadIdx.x * RS_DPT + j;
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; w++) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = (uint16_t)run;
                run += c;
            }
            tot[j] = run;
            sum += run;
        }
        uint32_t total;
        uint32_t excl = block_exclusive_scan<uint32_t>(sum, &total);
#pragma unroll
        for (int j = 0; j < RS_DPT; j++) {
            const int d = threadIdx.x * RS_DPT + j;
            dstart[d] = excl;
            excl += tot[j];
            gstart[d] = offsets[(size_t)d * tiles + blockIdx.x];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        if (dig[i] == RADIX) continue;
        const uint32_t pos = dstart[dig[i]] + wcnt[warp][dig[i]] + local[i];
        s_key[pos] = k[i];
        s_val[pos] = v[i];
    }
    __syncthreads();
    const uint32_t count = (uint32_t)min((size_t)RS_TILE, n - tile_base);
    for (uint32_t i = threadIdx.x; i < count; i += RS_THREADS) {
        const uint64_t key = s_key[i];
        const int d = (int)((key >> shift) & mask);
        const size_t pos = (size_t)gstart[d] + (i - dstart[d]);
        keys_out[pos] = key;
        vals_out[pos] = s_val[i];
    }
}

// The passes of the sort, ping-ponging between (keys, vals) and (kalt,
// valt); returns true when the result is left in (kalt, valt).
template <typename V>
bool radix_sort_passes(uint64_t *keys, V *vals, uint64_t *kalt, V *valt, size_t n, int begin_bit, int end_bit,
                       cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return false;
    if (n >= (size_t(1) << 32)) fail(TTC_ERR_RANGE, "radix sort: %zu elements exceed 2^32", n);
    const unsigned tiles = ceil_div(n, RS_TILE);
    DevBuf<uint32_t> counts((size_t)RADIX * tiles, s), offs((size_t)RADIX * tiles + 1, s);
    uint64_t *kin = keys, *kout = kalt;
    V *vin = vals, *vout = valt;
    const size_t dyn = (size_t)RS_TILE * (sizeof(uint64_t) + sizeof(V));
    ensure_smem((const void *)radix_scatter_kernel<V>, dyn);
    for (int shift = begin_bit; shift < end_bit; shift += RADIX_BITS) {
        const int width = std::min(RADIX_BITS, end_bit - shift);
        const uint32_t mask = (1u << width) - 1u;
        radix_hist_kernel<<<tiles, RS_THREADS, 0, s>>>(kin, n, shift, mask, counts.get(), tiles);
        TTC_LAUNCH_CHECK();
        exclusive_scan_impl<uint32_t, uint32_t>(counts.get(), offs.get(), (size_t)RADIX * tiles, s);
        radix_scatter_kernel<V><<<tiles, RS_THREADS, dyn, s>>>(kin, vin, kout, vout, n, shift, mask, offs.get(),
                                                               tiles);
        TTC_LAUNCH_CHECK();
        uint64_t *tk = kin; kin = kout; kout = tk;
        V *tv = vin; vin = vout; vout = tv;
    }
    return kin != keys;
}

template <typename V>
void radix_sort_impl(uint64_t *keys, V *vals, size_t n, int begin_bit, int end_bit, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return;
    DevBuf<uint64_t> kalt(n, s);
    DevBuf<V> valt(n, s);
    if (radix_sort_passes<V>(keys, vals, kalt.get(), valt.get(), n, begin_bit, end_bit, s)) {
        TTC_CUDA(cudaMemcpyAsync(keys, kalt.get(), n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        TTC_CUDA(cudaMemcpyAsync(vals, valt.get(), n * sizeof(V), cudaMemcpyDeviceToDevice, s));
    }
}

__global__ void minmax_kernel(const int64_t *in, size_t n, long long *dmin, long long *dmax) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const long long v = in[i];
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(dmin, lo);
        atomicMax(dmax, hi);
    }
}

__global__ void init_minmax_kernel(long long *dmin, long long *dmax) {
    *dmin = LLONG_MAX;
    *dmax = LLONG_MIN;
}

}  // namespace

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    exclusive_scan_impl<uint32_t, uint32_t>(in, out, n, s);
}
void exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, cudaStream_t s) {
    exclusive_scan_impl<uint64_t, uint64_t>(in, out, n, s);
}
void exclusive_scan_flags(const uint8_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    exclusive_scan_impl<uint32_t, uint8_t>(in, out, n, s);
}
void radix_sort_u64_u32(uint64_t *keys, uint32_t *vals, size_t n, int bits, cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, n, 0, bits, s);
}
void radix_sort_u64_u64(uint64_t *keys, uint64_t *vals, size_t n, int bits, cudaStream_t s) {
    radix_sort_impl<uint64_t>(keys, vals, n, 0, bits, s);
}
void radix_sort_u64_u64_range(uint64_t *keys, uint64_t *vals, size_t n, int begin_bit, int end_bit,
                              cudaStream_t s) {
    radix_sort_impl<uint64_t>(keys, vals, n, begin_bit, end_bit, s);
}
bool radix_sort_passes_u32(uint64_t *keys, uint32_t *vals, uint64_t *kalt, uint32_t *valt, size_t n, int begin_bit,
                           int end_bit, cudaStream_t s) {
    return radix_sort_passes<uint32_t>(keys, vals, kalt, valt, n, begin_bit, end_bit, s);
}
bool radix_sort_passes_u64(uint64_t *keys, uint64_t *vals, uint64_t *kalt, uint64_t *valt, size_t n, int begin_bit,
                           int end_bit, cudaStream_t s) {
    return radix_sort_passes<uint64_t>(keys, vals, kalt, valt, n, begin_bit, end_bit, s);
}
void reduce_minmax_i64(const int64_t *in, size_t n, int64_t *dmin, int64_t *dmax, cudaStream_t s) {
    init_minmax_kernel<<<1, 1, 0, s>>>((long long *)dmin, (long long *)dmax);
    TTC_LAUNCH_CHECK();
    if (!n) return;
    const unsigned blocks = (unsigned)(n < (size_t)sm_count() * 1024 ? ceil_div(n, 256) : (size_t)sm_count() * 4);
    minmax_kernel<<<blocks, 256, 0, s>>>(in, n, (long long *)dmin, (long long *)dmax);
    TTC_LAUNCH_CHECK();
}

}  // namespace ttc
