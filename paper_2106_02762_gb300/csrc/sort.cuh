// Stable radix sorts of device buffers that hand the result over by
// swapping buffers instead of copying it back (primitives.cu).
#pragma once

#include "common.cuh"

namespace ttc {

// The passes alone: sorts (keys, vals) with (kalt, valt) as scratch and
// returns true when the result is left in the scratch pair.
bool radix_sort_passes_u32(uint64_t *keys, uint32_t *vals, uint64_t *kalt, uint32_t *valt, size_t n, int begin_bit,
                           int end_bit, cudaStream_t s);
bool radix_sort_passes_u64(uint64_t *keys, uint64_t *vals, uint64_t *kalt, uint64_t *valt, size_t n, int begin_bit,
                           int end_bit, cudaStream_t s);
// Stable sort of buffer-held (key, value) pairs on key bits [begin_bit,
// end_bit) (64-bit keys; 32- or 64-bit values).  After an odd number of
// passes the scratch buffers hold the result and replace keys and vals, so
// nothing is copied back; raw pointers into the old buffers are then stale.
template <typename K, typename V>
void radix_sort_bufs(DevBuf<K> &keys, DevBuf<V> &vals, size_t n, int begin_bit, int end_bit, cudaStream_t s) {
    static_assert(sizeof(K) == 8 && (sizeof(V) == 4 || sizeof(V) == 8), "64-bit keys, 32- or 64-bit values");
    if (n <= 1 || end_bit <= begin_bit) return;
    // the scratch pair is as long as the buffers it may replace (a buffer
    // allocated with padding keeps it)
    DevBuf<K> kalt(keys.count > n ? keys.count : n, s);
    DevBuf<V> valt(vals.count > n ? vals.count : n, s);
    uint64_t *k0 = reinterpret_cast<uint64_t *>(keys.get()), *k1 = reinterpret_cast<uint64_t *>(kalt.get());
    bool alt;
    if constexpr (sizeof(V) == 4)
        alt = radix_sort_passes_u32(k0, reinterpret_cast<uint32_t *>(vals.get()), k1,
                                    reinterpret_cast<uint32_t *>(valt.get()), n, begin_bit, end_bit, s);
    else
        alt = radix_sort_passes_u64(k0, reinterpret_cast<uint64_t *>(vals.get()), k1,
                                    reinterpret_cast<uint64_t *>(valt.get()), n, begin_bit, end_bit, s);
    if (alt) {
        keys = static_cast<DevBuf<K> &&>(kalt);
        vals = static_cast<DevBuf<V> &&>(valt);
    }
}

}  // namespace ttc
