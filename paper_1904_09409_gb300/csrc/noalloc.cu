// ft_peaks_noalloc: the peak detection of ft_peaks for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc at the point where they detect peaks:
// code that records work into a CUDA graph through stream capture (allocation is
// not a capturable operation), services that reserve all device memory up front
// and forbid allocation afterwards, and hosts whose device memory is owned by
// another allocator.  ft_peaks keeps its per-tile key buffer in the plan's
// workspace, which it may grow with cudaMalloc.  This entry point instead uses
// the fixed array below, which the library image holds on every GPU that loads
// it until the process exits, and needs no plan at all.
#include <mutex>

#include "ft_internal.cuh"

#define FT_NOALLOC_MAX_DEVICES 64

// Scratch for the per-tile keys and one running bound per map.  Every call
// writes all the key slots it reads (padding included) and clears the bounds
// with cudaMemsetAsync on its stream before use, so stale contents from an
// earlier call never matter.  All calls share this one array: calls whose work
// overlaps on the GPU (other streams, or other host threads) race on it.
static __device__ __align__(256) unsigned char g_peak_scratch[FT_NOALLOC_SCRATCH_BYTES];

static std::mutex g_setup_mutex;
static void* g_scratch_addr[FT_NOALLOC_MAX_DEVICES];

// Device address of g_peak_scratch on the current device, looked up once per
// device.  In host code the symbol names a host-side stand-in, so the address
// must come from cudaGetSymbolAddress with the device current.
static cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= FT_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_peak_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

extern "C" ft_status ft_peaks_noalloc(const float* d_map, int n_intercept, int n_slope, int batch,
                                      int top_k, float threshold, ft_peak* d_out, int32_t* d_count,
                                      void* stream) {
    if (batch < 0 || batch > 65535 || top_k < 1 || top_k > FT_MAX_TOPK || threshold != threshold)
        return FT_ERR_INVALID_ARG;
    if (n_intercept < 2 || n_slope < 2) return FT_ERR_UNSUPPORTED_SIZE;
    if ((long long)n_intercept * n_slope > 0xFFFFFFFFll) return FT_ERR_UNSUPPORTED_SIZE;
    if (batch == 0) return FT_OK;
    if (!d_map || !d_out || !d_count) return FT_ERR_INVALID_ARG;
    if (peaks_key_bytes(n_intercept, n_slope, batch, top_k) > (size_t)FT_NOALLOC_SCRATCH_BYTES)
        return ft_record_error(FT_ERR_UNSUPPORTED_SIZE,
                               "ft_peaks_noalloc: batch x tiles x top_k keys exceed the fixed scratch "
                               "of FT_NOALLOC_SCRATCH_BYTES");
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_peaks_noalloc: cudaGetSymbolAddress");
    unsigned long long* keys = (unsigned long long*)scratch;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* bounds = peaks_bounds(keys, n_intercept, n_slope, batch, top_k);
    e = launch_peak_tiles(d_map, n_intercept, n_slope, batch, top_k, threshold, keys, bounds, st);
    if (e == cudaSuccess)
        e = launch_peak_select(keys, bounds, n_intercept, n_slope, batch, top_k, d_out, d_count, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_peaks_noalloc: launch");
    return FT_OK;
}
