// Mixed-size batches in one launch per stage (the paper's Sec. I remark that the
// rows and columns of the transform are independent, taken across images of
// uneven sizes).
//
// Each stage of Sec. 3.1 (step 1, steps 2-3, step 4) and the peak pass of
// Sec. 4.4 is one persistent kernel over every image of the batch, whatever its
// size: resident blocks take (image, block) items from a device work queue (one
// atomic counter per stage) and run the fixed-length block of fast_blocks.cuh
// for that image's length, chosen by a switch on the length.  The threads per
// block are fixed per launch (the autotuner's knob for each stage), so the
// transforms per block follow from the length: B = threads / fs_T(length), and
// every item holds the same number of samples (E x threads), whatever its image.
// Items are listed largest image first, so the queue ends on small items.  A
// stage waits for nothing but its own items: the kernel boundary orders the
// stages, and no block ever waits on another.
#include "fast_blocks.cuh"
#include "peak_sparse_block.cuh"

#define FT_BATCH_LENGTHS(X) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)

// Run body(i) for every item i the block takes from the queue: thread 0 fetches
// the next index while the block works on the current one.  Every thread of the
// block must call it.
template <typename Body>
__device__ __forceinline__ void run_queue(unsigned* queue, int nitems, Body body) {
    __shared__ int slot[2];
    if (threadIdx.x == 0) slot[0] = (int)atomicAdd(queue, 1u);
    __syncthreads();
    for (int k = 0;; k ^= 1) {
        const int i = slot[k];
        if (i >= nitems) break;                        // the same index for the whole block
        if (threadIdx.x == 0) slot[k ^ 1] = (int)atomicAdd(queue, 1u);
        body(i);
        __syncthreads();                               // shared memory and slot[k] are free again
    }
}

// step 1: column block it.y of image it.x
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_batch_r2c(const BatchImg* __restrict__ imgs, const int2* __restrict__ items, int nitems, unsigned* __restrict__ queue,
            const float* __restrict__ in, float2* __restrict__ ws) {
    extern __shared__ float2 sm[];
    run_queue(queue, nitems, [&](int i) {
        const int2 it = items[i];
        const BatchImg& d = imgs[it.x];
        const int W = d.W;
        const float* src = in + d.img_off;
        float2* dst = ws + d.ws_off;
        switch (d.H) {
#define X(n) case n: r2c_block<n, NT / fs_T(n)>(src, n, W, W, 0, d.stw_y, dst, W, 1.f, 1.f, it.y, sm); break;
            FT_BATCH_LENGTHS(X)
#undef X
        }
    });
}

// steps 2-3: row block it.y of image it.x (n_slope = W)
template <int NT, int INTERP>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_batch_rows(const BatchImg* __restrict__ imgs, const int2* __restrict__ items, int nitems,
             unsigned* __restrict__ queue, float2* __restrict__ ws) {
    extern __shared__ float2 sm[];
    run_queue(queue, nitems, [&](int i) {
        const int2 it = items[i];
        const BatchImg& d = imgs[it.x];
        const int H = d.H;
        float2* base = ws + d.ws_off;
        switch (d.W) {
#define X(n) case n: rows_block<n, INTERP, NT / fs_T(n)>(base, n, H, H / 2 + 1, d.stw_x, it.y, sm); break;
            FT_BATCH_LENGTHS(X)
#undef X
        }
    });
}

// step 4 with the tile maxima of |map|: column block it.y of image it.x
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_batch_c2r(const BatchImg* __restrict__ imgs, const int2* __restrict__ items, int nitems, unsigned* __restrict__ queue,
            const float2* __restrict__ ws, float* __restrict__ maps, unsigned* __restrict__ tmax) {
    extern __shared__ float2 sm[];
    run_queue(queue, nitems, [&](int i) {
        const int2 it = items[i];
        const BatchImg& d = imgs[it.x];
        const int W = d.W;
        const float2* src = ws + d.ws_off;
        float* dst = maps + d.map_off;
        unsigned* tm = tmax ? tmax + d.tm_off : nullptr;
        switch (d.H) {
#define X(n)                                                                                                  \
    case n: {                                                                                                 \
        constexpr int B = NT / fs_T(n);                                                                       \
        c2r_block<n, B>(src, W, W, d.stw_y, 1.f, dst, 0, n, W, 1.f / (float)n, tm, (W + 2 * B - 1) / (2 * B), \
                        it.y, sm);                                                                            \
    } break;
            FT_BATCH_LENGTHS(X)
#undef X
        }
    });
}

// Sec. 4.4 from step 4's tile maxima, one image per item
__global__ void __launch_bounds__(1024)
k_batch_peaks(const BatchImg* __restrict__ imgs, int nimg, unsigned* __restrict__ queue, const float* __restrict__ maps,
              const unsigned* __restrict__ tmax, int c2r_threads, int K, float thr, ft_peak* __restrict__ out,
              int32_t* __restrict__ count) {
    extern __shared__ __align__(16) unsigned char spsm[];
    __shared__ SparseShared sh;
    run_queue(queue, nimg, [&](int j) {
        const BatchImg& d = imgs[j];
        const int H = d.H, W = d.W;
        const int B = c2r_threads / fs_T(H);
        const int TH = 128 / B, TW = 2 * B;
        int logTW = 0;
        while ((1 << logTW) < TW) ++logTW;
        peak_sparse_block(maps + d.map_off, tmax + d.tm_off, H, W, TH, logTW, H / TH, (W + TW - 1) / TW, K, thr,
                          out + (size_t)d.pos * K, count + d.pos, spsm, sh);
    });
}

// ---------------------------------------------------------------- host side
bool batch_threads_ok(int stage, int threads) {
    if (stage == 1) return threads == 128 || threads == 256;
    return threads == 256 || threads == 512;
}

int batch_r2c_blocks(int H, int W, int threads) {
    const int B = threads / fs_T(H);
    return (W + 2 * B - 1) / (2 * B);
}
int batch_rows_blocks(int H, int W, int threads) {
    const int B = threads / fs_T(W);
    return (H / 2 + 1 + B - 1) / B;
}
int batch_c2r_blocks(int H, int W, int threads) { return batch_r2c_blocks(H, W, threads); }

void batch_tile_shape(int H, int W, int threads, int* rows, int* cols, int* bands, int* nbx) {
    const int B = threads / fs_T(H);
    *rows = 128 / B;
    *cols = 2 * B;
    *bands = H / *rows;
    *nbx = (W + 2 * B - 1) / (2 * B);
}

// shared memory of the transform stages: the exchange buffer of B = threads / T
// transforms (and, for the rows, B staged rows of W + 4 samples), the largest
// over the lengths up to maxlen
static size_t stage_smem(int stage, int threads, int maxlen) {
    size_t best = 0;
    for (int n : {128, 192, 256, 384, 512, 768, 1024, 1536, 2048}) {
        if (n > maxlen) continue;
        const int B = threads / fs_T(n);
        size_t v = (size_t)fs_slots(n) * B;
        if (stage == 1 && (size_t)srow_pitch(n) * B > v) v = (size_t)srow_pitch(n) * B;
        if (v * sizeof(float2) > best) best = v * sizeof(float2);
    }
    return best;
}

template <typename K>
static cudaError_t persistent_launch(K kernel, int threads, size_t sm, int nitems, cudaStream_t st, dim3* grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, sm)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int g = sms * per;
    *grid = dim3(nitems < g ? nitems : g);
    return cudaSuccess;
}

cudaError_t launch_batch_r2c(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, const float* in,
                             float2* ws, int threads, int maxH, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const size_t sm = stage_smem(0, threads, maxH);
    dim3 g;
    cudaError_t e;
    if (threads == 256) {
        if ((e = persistent_launch(k_batch_r2c<256>, 256, sm, nitems, st, &g)) != cudaSuccess) return e;
        k_batch_r2c<256><<<g, 256, sm, st>>>(imgs, items, nitems, queue, in, ws);
    } else if (threads == 512) {
        if ((e = persistent_launch(k_batch_r2c<512>, 512, sm, nitems, st, &g)) != cudaSuccess) return e;
        k_batch_r2c<512><<<g, 512, sm, st>>>(imgs, items, nitems, queue, in, ws);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NT>
static cudaError_t go_rows(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, float2* ws,
                           int interp, size_t sm, cudaStream_t st) {
    dim3 g;
    cudaError_t e;
    if (interp == FT_INTERP_LINEAR) {
        if ((e = persistent_launch(k_batch_rows<NT, FT_INTERP_LINEAR>, NT, sm, nitems, st, &g)) != cudaSuccess)
            return e;
        k_batch_rows<NT, FT_INTERP_LINEAR><<<g, NT, sm, st>>>(imgs, items, nitems, queue, ws);
    } else {
        if ((e = persistent_launch(k_batch_rows<NT, FT_INTERP_CUBIC>, NT, sm, nitems, st, &g)) != cudaSuccess)
            return e;
        k_batch_rows<NT, FT_INTERP_CUBIC><<<g, NT, sm, st>>>(imgs, items, nitems, queue, ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_rows(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, float2* ws,
                              int interp, int threads, int maxW, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (interp != FT_INTERP_LINEAR && interp != FT_INTERP_CUBIC) return cudaErrorInvalidValue;
    const size_t sm = stage_smem(1, threads, maxW);
    if (threads == 128) return go_rows<128>(imgs, items, nitems, queue, ws, interp, sm, st);
    if (threads == 256) return go_rows<256>(imgs, items, nitems, queue, ws, interp, sm, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_c2r(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, const float2* ws,
                             float* maps, unsigned* tmax, int threads, int maxH, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const size_t sm = stage_smem(2, threads, maxH);
    dim3 g;
    cudaError_t e;
    if (threads == 256) {
        if ((e = persistent_launch(k_batch_c2r<256>, 256, sm, nitems, st, &g)) != cudaSuccess) return e;
        k_batch_c2r<256><<<g, 256, sm, st>>>(imgs, items, nitems, queue, ws, maps, tmax);
    } else if (threads == 512) {
        if ((e = persistent_launch(k_batch_c2r<512>, 512, sm, nitems, st, &g)) != cudaSuccess) return e;
        k_batch_c2r<512><<<g, 512, sm, st>>>(imgs, items, nitems, queue, ws, maps, tmax);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t batch_peaks_smem(const BatchImg* host_imgs, int nimg, int c2r_threads, int top_k) {
    size_t best = 0;
    for (int j = 0; j < nimg; ++j) {
        int rows, cols, bands, nbx;
        batch_tile_shape(host_imgs[j].H, host_imgs[j].W, c2r_threads, &rows, &cols, &bands, &nbx);
        const size_t v = sparse_smem(rows, cols, top_k, 32, bands * nbx);
        if (v > best) best = v;
    }
    return best;
}

cudaError_t launch_batch_peaks(const BatchImg* imgs, int nimg, unsigned* queue, const float* maps, const unsigned* tmax,
                               int c2r_threads, int top_k, float threshold, ft_peak* out, int32_t* count, size_t smem,
                               cudaStream_t st) {
    if (nimg <= 0) return cudaSuccess;
    dim3 g;
    cudaError_t e = persistent_launch(k_batch_peaks, 1024, smem, nimg, st, &g);
    if (e != cudaSuccess) return e;
    k_batch_peaks<<<g, 1024, smem, st>>>(imgs, nimg, queue, maps, tmax, c2r_threads, top_k, threshold, out, count);
    return cudaGetLastError();
}
