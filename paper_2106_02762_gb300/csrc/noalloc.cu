// ttc_count_noalloc: one query without any device allocation.
//
// Some callers cannot allocate device memory at the moment they count: hosts
// whose framework's caching allocator owns nearly all of HBM and forbids
// foreign allocations, and latency-critical loops where an allocation can
// stall or synchronise the device.  This entry point serves them: it runs the
// same light and prefix-sum kernels as ttc_count, but every device buffer it
// needs beyond the graph and the caller's output lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded.  The
// call is synchronous: it waits for its kernels and copies the counts back
// before it returns.
#include <cstring>
#include <mutex>

#include "graph.cuh"

namespace ttc {
void set_last_error(const std::string &m);
void normalise(const ttc_delta &d, int64_t out[3]);
}  // namespace ttc

using namespace ttc;

namespace {

// Layout: [0, 256) counts (8 u64) + overflow flag; [256, 512) the normalised
// delta-triple; [512, end) the prefix arrays of the heavy (CEC) path.
constexpr size_t NOALLOC_HEAD = 512;
static __device__ __align__(256) unsigned char g_noalloc_scratch[TTC_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;             // one call at a time per process
void *g_noalloc_ptr[MAX_DEVICES] = {};  // device address of the array, per device

// Device address of the array on the current device (set-up on first use).
void *noalloc_base(int dev) {
    if (dev < 0 || dev >= MAX_DEVICES) fail(TTC_ERR_INVALID, "device %d out of range", dev);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(TTC_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" ttc_status ttc_count_noalloc(ttc_graph *g, const ttc_delta *d, uint64_t out[TTC_NUM_TYPES],
                                        void *stream) {
    if (!g || !d || !out) {
        set_last_error("NULL argument");
        return TTC_ERR_INVALID;
    }
    if (g->streamed) {
        set_last_error("the graph was loaded with TTC_LOAD_STREAM, whose counts need scratch of their own");
        return TTC_ERR_INVALID;
    }
    try {
        int64_t hq[3];
        normalise(*d, hq);
        const size_t need = heavy_scratch_bytes(g);
        if (need > TTC_NOALLOC_SCRATCH_BYTES - NOALLOC_HEAD)
            fail(TTC_ERR_RANGE,
                 "graph needs %zu bytes of prefix scratch; ttc_count_noalloc holds %zu (use ttc_count)", need,
                 (size_t)(TTC_NOALLOC_SCRATCH_BYTES - NOALLOC_HEAD));
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        int caller_dev = 0;
        TTC_CUDA(cudaGetDevice(&caller_dev));
        // the caller's current device is current again whenever this returns
        struct Restore {
            int dev;
            ~Restore() { cudaSetDevice(dev); }
        } restore{caller_dev};
        TTC_CUDA(cudaSetDevice(g->device));
        cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g->stream;
        unsigned char *base = static_cast<unsigned char *>(noalloc_base(g->device));
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(base);
        int64_t *dq = reinterpret_cast<int64_t *>(base + 256);
        // the counts and the overflow flag must start at zero; the prefix
        // region is written in full by the kernels before it is read
        TTC_CUDA(cudaMemsetAsync(acc, 0, 9 * sizeof(unsigned long long), s));
        TTC_CUDA(cudaMemcpyAsync(dq, hq, sizeof hq, cudaMemcpyHostToDevice, s));
        count_one_into(g, dq, acc, base + NOALLOC_HEAD, s);
        unsigned long long h[9];
        TTC_CUDA(cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, s));
        TTC_CUDA(cudaStreamSynchronize(s));
        check_count_flag(h[8]);
        memcpy(out, h, 8 * sizeof(uint64_t));
        return TTC_OK;
    } catch (const Failure &f) {
        set_last_error(f.message);
        return f.status;
    } catch (...) {
        set_last_error("unexpected internal failure");
        return TTC_ERR_INTERNAL;
    }
}
