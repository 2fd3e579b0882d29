// pod_sample_noalloc: the column draw step (same kernel as pod_sample) with
// its scratch in fixed-size device arrays declared in this file, so that the
// call makes no device allocation.
//
// Who needs it: callers that may not or cannot allocate device memory at the
// moment they draw -- a process whose device memory pool is capped or already
// fully reserved by another framework, or a latency-critical loop that must
// not touch the allocator.  Such callers pass their own inputs and outputs
// and get the scratch from these arrays instead of from cudaMalloc.  The call
// itself issues CUDA API calls (an address lookup, copies, a launch), so it
// must not be made from a host callback (cudaLaunchHostFunc,
// cudaStreamAddCallback), where CUDA forbids API calls.
//
// The arrays live in every GPU that loads this library, for the life of the
// process (about 1.1 MB each).  With CUDA's lazy module loading they are
// placed in device memory when this file's device code is first used, which
// is the first call's address lookup: make one call per device at set-up,
// while allocating is still possible.  All calls share the arrays: two calls
// that overlap on the GPU (different streams, or different host threads on
// one device) race on the scratch and must be serialised by the caller.
#include <mutex>

#include "pod_internal.h"

namespace {

constexpr int64_t NOALLOC_MAX_N = 1 << 16;   // columns
constexpr int NOALLOC_MAX_C = 4096;          // draws
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) uint64_t g_na_w[NOALLOC_MAX_N];
static __device__ __align__(256) uint64_t g_na_cdf[NOALLOC_MAX_N];
static __device__ __align__(256) uint8_t g_na_flags[NOALLOC_MAX_N];
static __device__ __align__(256) int32_t g_na_draws[NOALLOC_MAX_C];

struct DevScratch {
    bool ready;
    uint64_t *w, *cdf;
    uint8_t *flags;
    int32_t *draws;
};

DevScratch g_scratch[NOALLOC_MAX_DEVICES];
std::mutex g_scratch_mu;

// Device addresses of the arrays for the current device.  The first call on
// a device looks them up with cudaGetSymbolAddress (host code cannot use the
// arrays' names as device pointers); later calls reuse the cached values.
pod_status scratch_for_current_device(DevScratch *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return POD_ECUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return POD_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DevScratch &s = g_scratch[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_w) != cudaSuccess) { cudaGetLastError(); return POD_ECUDA; }
        s.w = (uint64_t *)p;
        if (cudaGetSymbolAddress(&p, g_na_cdf) != cudaSuccess) { cudaGetLastError(); return POD_ECUDA; }
        s.cdf = (uint64_t *)p;
        if (cudaGetSymbolAddress(&p, g_na_flags) != cudaSuccess) { cudaGetLastError(); return POD_ECUDA; }
        s.flags = (uint8_t *)p;
        if (cudaGetSymbolAddress(&p, g_na_draws) != cudaSuccess) { cudaGetLastError(); return POD_ECUDA; }
        s.draws = (int32_t *)p;
        s.ready = true;
    }
    *out = s;
    return POD_OK;
}

}  // namespace

extern "C" pod_status pod_sample_noalloc(const uint64_t *w_dev, uint8_t *mask_dev, int64_t n, int32_t c,
                                         uint64_t seed, int32_t t, int32_t stream_id, int32_t *idx_dev,
                                         int32_t *g_dev, void *stream) {
    if (!w_dev || !mask_dev || !idx_dev || !g_dev || n <= 0 || c <= 0 || t < 0 || stream_id < 0)
        return POD_EINVAL;
    if (n > NOALLOC_MAX_N || c > NOALLOC_MAX_C) return POD_EUNSUPPORTED;
    DevScratch s{};
    POD_TRY(scratch_for_current_device(&s));
    cudaStream_t st = (cudaStream_t)stream;
    // the arrays keep whatever the previous call left: copy the weights in
    // and clear the flags the draw kernel expects to start at zero
    POD_CUDA_TRY(cudaMemcpyAsync(s.w, w_dev, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    POD_CUDA_TRY(cudaMemsetAsync(s.flags, 0, (size_t)n, st));
    SampleArgs a{};
    a.n = n;
    a.c = c;
    a.mode_round0 = 3;
    a.mode = 3;
    a.seed = seed;
    a.stream_id = stream_id;
    a.w = s.w;
    a.cdf = s.cdf;
    a.mask = mask_dev;
    a.flags = s.flags;
    a.draws = s.draws;
    a.idx = idx_dev;
    a.st = nullptr;
    a.g_out = g_dev;
    a.t_fixed = t;
    return launch_sample(a, st);
}
