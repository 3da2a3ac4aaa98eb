// Shared host/device plumbing for the ttc library: error propagation,
// stream-ordered device buffers, and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ttc.h"

namespace ttc {

// Internal failures travel as exceptions and become a ttc_status at the C
// boundary (capi.cu).
struct Failure {
    ttc_status status;
    std::string message;
};

[[noreturn]] void fail(ttc_status st, const char *fmt, ...);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define TTC_CUDA(call) ::ttc::cuda_check((call), #call, __FILE__, __LINE__)
void note_launch();
#define TTC_LAUNCH_CHECK() \
    (::ttc::note_launch(), ::ttc::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))

// Device allocation through the stream-ordered allocator, with the testing
// hook that fails the n-th allocation.
void *device_alloc(size_t bytes, cudaStream_t s);
void device_free(void *p, cudaStream_t s);
cudaMemPool_t library_pool();
uint64_t pool_cached_bytes();
uint64_t device_bytes_in_use();

template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t count = 0;
    cudaStream_t stream = 0;
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t s) { alloc(n, s); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { *this = static_cast<DevBuf &&>(o); }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            reset();
            ptr = o.ptr; count = o.count; stream = o.stream;
            o.ptr = nullptr; o.count = 0;
        }
        return *this;
    }
    ~DevBuf() { reset(); }
    void alloc(size_t n, cudaStream_t s) {
        reset();
        stream = s;
        count = n;
        ptr = static_cast<T *>(device_alloc(sizeof(T) * (n ? n : 1), s));
    }
    void reset() {
        if (ptr) device_free(ptr, stream);
        ptr = nullptr;
        count = 0;
    }
    size_t bytes() const { return sizeof(T) * count; }
    T *get() const { return ptr; }
};

// Number of SMs of the current device (cached per device).
int sm_count();

// Raises kernel `fn`'s dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device, size); thread-safe.
void ensure_smem(const void *fn, size_t bytes);

// While an object of this type lives, the calling thread's count calls
// record no per-kernel timing (the handle's profiling setting is left as it
// is, so other threads see no change).
struct ProfOff {
    ProfOff();
    ~ProfOff();
    ProfOff(const ProfOff &) = delete;
    ProfOff &operator=(const ProfOff &) = delete;
};

// ---------------------------------------------------------------- primitives
// (primitives.cu)  All run on stream `s` and use scratch from DevBuf.

// out[i] = sum of in[0..i) for i in [0, n]; returns nothing (out has n+1 slots).
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s);
void exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, cudaStream_t s);
// Same, but the input is an array of 0/1 bytes.
void exclusive_scan_flags(const uint8_t *in, uint32_t *out, size_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).  Sorts in
// place: keys/vals hold the result on return (alt buffers are scratch).
void radix_sort_u64_u32(uint64_t *keys, uint32_t *vals, size_t n, int bits, cudaStream_t s);
void radix_sort_u64_u64(uint64_t *keys, uint64_t *vals, size_t n, int bits, cudaStream_t s);
// Stable sort on key bits [begin_bit, end_bit) only.
void radix_sort_u64_u64_range(uint64_t *keys, uint64_t *vals, size_t n, int begin_bit, int end_bit,
                              cudaStream_t s);

// Reductions into a device scalar (the caller copies it back).
void reduce_minmax_i64(const int64_t *in, size_t n, int64_t *dmin, int64_t *dmax, cudaStream_t s);

inline int bits_for(uint64_t x) {  // bits needed to store values 0..x
    int b = 0;
    while (b < 64 && (x >> b) != 0) b++;
    return b;
}

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace ttc
