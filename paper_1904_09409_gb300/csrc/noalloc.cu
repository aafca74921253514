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
#include <cuda.h>

#include <mutex>

#include "ft_internal.cuh"

#define FT_NOALLOC_CACHE 64

// Scratch for the per-tile keys and one running bound per map.  Every call
// writes all the key slots it reads (padding included) and clears the bounds
// with cudaMemsetAsync on its stream before use, so stale contents from an
// earlier call never matter.  All calls share this one array: calls whose work
// overlaps on the GPU (other streams, or other host threads) race on it.
static __device__ __align__(256) unsigned char g_peak_scratch[FT_NOALLOC_SCRATCH_BYTES];

// The array's device address belongs to the module loaded in one CUDA context:
// a cudaDeviceReset, or another context made current on the same device, gives
// it another address.  The cache is therefore keyed by the context's unique id
// (cuCtxGetId, never reused within a process), not by the device ordinal.
typedef CUresult (*ctx_current_fn)(CUcontext*);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long*);

static std::mutex g_setup_mutex;
static ctx_current_fn g_ctx_current = nullptr;
static ctx_id_fn g_ctx_id = nullptr;
static unsigned long long g_cache_ctx[FT_NOALLOC_CACHE];
static void* g_cache_addr[FT_NOALLOC_CACHE];
static int g_cache_next = 0;

// Id of the current context (the device's primary context is created first if
// no context is current).  Host-side queries only: no stream work, so it is
// also safe while a stream is being captured.
static cudaError_t current_context_id(unsigned long long* id) {
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_ctx_current || !g_ctx_id) {
            cudaDriverEntryPointQueryResult q1, q2;
            void *f1 = nullptr, *f2 = nullptr;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
            if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
            if (e != cudaSuccess) return e;
            if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
                return cudaErrorNotSupported;
            g_ctx_current = (ctx_current_fn)f1;
            g_ctx_id = (ctx_id_fn)f2;
        }
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);      // creates the primary context
        if (e != cudaSuccess) return e;
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    }
    return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of g_peak_scratch in the current context, looked up once per
// context.  In host code the symbol names a host-side stand-in, so the address
// must come from cudaGetSymbolAddress with that context current.
static cudaError_t scratch_address(void** out) {
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    for (int i = 0; i < FT_NOALLOC_CACHE; ++i)
        if (g_cache_addr[i] && g_cache_ctx[i] == id) {
            *out = g_cache_addr[i];
            return cudaSuccess;
        }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_peak_scratch);
    if (e != cudaSuccess) return e;
    g_cache_ctx[g_cache_next] = id;
    g_cache_addr[g_cache_next] = p;
    g_cache_next = (g_cache_next + 1) % FT_NOALLOC_CACHE;
    *out = p;
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
