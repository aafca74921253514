// Fixed-length versions of the column and row kernels over a uniform batch
// (see k_cols.cu and k_rows.cu for what each step computes): one block of
// fast_blocks.cuh per CUDA block, the image index in blockIdx.y.
#include <string.h>

#include "fast_blocks.cuh"

// tma_nb > 0: the image columns are staged by tma_nb tensor copies of tma_h
// rows (tmap describes the launch's images), else read from global memory.
// follows_peak: the predecessor on the stream is the peak pass of the previous
// batch of ft_detect_batches, which has waited for its own step 4 and touches
// only the maps, the tile maxima and the peak records: this kernel reads its
// images and writes the spectrum workspace without waiting for it, and only its
// last block waits for that pass before exiting, so that the completion of this
// grid (which the next kernels wait for) implies the completion of the pass.
template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bcol(N), 1024 / (fs_T(N) * fs_Bcol(N)))
k_col_r2c_fast(const float* __restrict__ in, int rows_in, int ncols, int in_pitch, size_t in_img,
               int row0, const float2* __restrict__ stw, float2* __restrict__ out, int out_pitch,
               size_t out_img, float end_scale, float mid_scale, const __grid_constant__ CUtensorMap tmap,
               int tma_h, int tma_nb, unsigned* __restrict__ err, long long wait, int pf, int follows_peak) {
    extern __shared__ __align__(128) float2 sm[];
    pdl_trigger();
    if (!follows_peak) pdl_wait();
    const float* src = in + (size_t)blockIdx.y * in_img;
    float2* dst = out + (size_t)blockIdx.y * out_img;
    if (tma_nb > 0) {
        const int nxt = blockIdx.y * gridDim.x + blockIdx.x + pf;
        const int pimg = pf > 0 && nxt < gridDim.x * gridDim.y ? nxt / gridDim.x : -1;
        r2c_block<N, fs_Bcol(N), true>(src, rows_in, ncols, in_pitch, row0, stw, dst, out_pitch, end_scale,
                                       mid_scale, blockIdx.x, sm, &tmap, tma_h, tma_nb, blockIdx.y, err, wait,
                                       nxt - pimg * gridDim.x, pimg);
    }
    else
        r2c_block<N, fs_Bcol(N)>(src, rows_in, ncols, in_pitch, row0, stw, dst, out_pitch, end_scale, mid_scale,
                                 blockIdx.x, sm);
    if (follows_peak && blockIdx.x == gridDim.x - 1 && blockIdx.y == gridDim.y - 1) pdl_wait();
}

// tma_nb > 0: the Hermitian half is staged by tma_nb tensor copies of tma_h rows
// (tmap describes the launch's half spectra), else by cp.async
template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bc2r(N), 1024 / (fs_T(N) * fs_Bc2r(N)))
k_col_c2r_fast(const float2* __restrict__ in, int ncols, int in_pitch, size_t in_img,
               const float2* __restrict__ stw, float mid_scale, float* __restrict__ out, int row0,
               int rows_out, int out_pitch, size_t out_img, float out_scale, unsigned* __restrict__ tmax,
               const __grid_constant__ CUtensorMap tmap, int tma_h, int tma_nb, unsigned* __restrict__ err,
               long long wait, int pf) {
    extern __shared__ __align__(128) float2 sm[];
    pdl_trigger();
    pdl_wait();
    constexpr int bands = fs_E(N) * fs_T(N) / c2r_tile_rows(N);
    const float2* src = in + (size_t)blockIdx.y * in_img;
    float* dst = out + (size_t)blockIdx.y * out_img;
    unsigned* tm = tmax ? tmax + (size_t)blockIdx.y * bands * gridDim.x : nullptr;
    if (tma_nb > 0) {
        const int nxt = blockIdx.y * gridDim.x + blockIdx.x + pf;
        const int pimg = pf > 0 && nxt < gridDim.x * gridDim.y ? nxt / gridDim.x : -1;
        c2r_block<N, fs_Bc2r(N), true>(src, ncols, in_pitch, stw, mid_scale, dst, row0, rows_out, out_pitch,
                                       out_scale, tm, gridDim.x, blockIdx.x, sm, &tmap, tma_h, tma_nb, blockIdx.y,
                                       err, wait, nxt - pimg * gridDim.x, pimg);
    }
    else
        c2r_block<N, fs_Bc2r(N)>(src, ncols, in_pitch, stw, mid_scale, dst, row0, rows_out, out_pitch, out_scale,
                                 tm, gridDim.x, blockIdx.x, sm);
}

// The adjoint of step 4 fed straight from the loss of the gradient workload:
// the input column pair is not a stored gradient map but
//     g = 2 r scale sign(P) gscale,   r = |P| scale - T
// computed from the map P and the target T as the columns are loaded (the loss
// gradient of k_loss.cu), while every thread adds r^2 of its samples (FP32,
// compensated) and the block writes one partial of the image's loss.  Each map
// cell is loaded by exactly one thread, so the partials of an image's blocks
// add up to its sum of r^2 (within a block by a fixed shuffle tree).  With
// tma_nb > 0 the map columns arrive by tensor copies into the exchange buffer
// (pmap, waited for with the bound `wait`; bit 3 of *err when it runs out, and
// the block returns without writing), their values go to registers, and the
// target columns (tmapt) follow into the same buffer; the map and target boxes
// of the block pf blocks later are prefetched into L2.  Everything after the
// load is r2c_finish.
template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bcol(N), 1024 / (fs_T(N) * fs_Bcol(N)))
k_col_r2c_loss_fast(const float* __restrict__ map, const float* __restrict__ target, int ncols, size_t img_cells,
                    const float2* __restrict__ stw, float2* __restrict__ out, int out_pitch, size_t out_img,
                    float end_scale, float mid_scale, float scale, float gscale, float* __restrict__ partial,
                    const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap tmapt, int tma_h,
                    int tma_nb, unsigned* __restrict__ err, long long wait, int pf) {
    constexpr int B = fs_Bcol(N), E = fs_E(N), NT = fs_T(N) * fs_Bcol(N), NW = NT / 32;
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    using F = FastFft<N, -1, B>;
    extern __shared__ __align__(128) float2 sm[];
    __shared__ float red[NW];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = blockIdx.x * 2 * B + 2 * f;
    const bool colok = c < ncols;
    const float* P = map + (size_t)blockIdx.y * img_cells + c;
    const float* Tg = target + (size_t)blockIdx.y * img_cells + c;
    const float* stg = reinterpret_cast<const float*>(sm);   // [tma_nb tma_h][2B] map, then target values
    __shared__ uint64_t mbar;
    const uint32_t mb = smem_u32(&mbar);
    float2 v[E];
    if (tma_nb > 0) {
        // the block's map columns by tensor copies into the exchange buffer, their
        // values to registers, then the target columns into the same buffer
        // (the mbarrier's second phase; both are read before the FFT's first
        // exchange); the map and target boxes of the block pf blocks later are
        // prefetched into L2
        if (threadIdx.x == 0) {
            mbar_init(mb, 1);
            mbar_arrive_expect_tx(mb, (uint32_t)(tma_nb * tma_h * 2 * B * sizeof(float)));
            for (int k = 0; k < tma_nb; ++k)
                tma_load_3d(reinterpret_cast<float*>(sm) + k * tma_h * 2 * B, &pmap, blockIdx.x * 2 * B, k * tma_h,
                            blockIdx.y, mb);
            const int nxt = blockIdx.y * gridDim.x + blockIdx.x + pf;
            if (pf > 0 && nxt < gridDim.x * gridDim.y) {
                const int pimg = nxt / gridDim.x, pbx = nxt - pimg * gridDim.x;
                for (int k = 0; k < tma_nb; ++k) {
                    tma_prefetch_3d(&pmap, pbx * 2 * B, k * tma_h, pimg);
                    tma_prefetch_3d(&tmapt, pbx * 2 * B, k * tma_h, pimg);
                }
            }
        }
        __syncthreads();                               // the mbarrier is initialised
        bool ok = mbar_wait(mb, 0, wait);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && err) atomicOr(err, 8u);
            mbar_wait(mb, 0);                          // the copies in flight land first
            return;
        }
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q)
                v[m * R0 + q] = *reinterpret_cast<const float2*>(stg + F::template in_pos<0>(t, m, q) * 2 * B + 2 * f);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // these reads before the refill
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(mb, (uint32_t)(tma_nb * tma_h * 2 * B * sizeof(float)));
            for (int k = 0; k < tma_nb; ++k)
                tma_load_3d(reinterpret_cast<float*>(sm) + k * tma_h * 2 * B, &tmapt, blockIdx.x * 2 * B, k * tma_h,
                            blockIdx.y, mb);
        }
        ok = mbar_wait(mb, 1, wait);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && err) atomicOr(err, 8u);
            mbar_wait(mb, 1);
            return;
        }
    }

    float acc = 0.f, comp = 0.f;
    auto add = [&](float y) {                          // compensated sum of r^2
        const float z = y - comp;
        const float s2 = acc + z;
        comp = (s2 - acc) - z;
        acc = s2;
    };
#pragma unroll
    for (int m = 0; m < G0; ++m)
#pragma unroll
        for (int q = 0; q < R0; ++q) {
            const int row = F::template in_pos<0>(t, m, q);
            float2 g = make_float2(0.f, 0.f);
            if (colok) {
                const float2 p = tma_nb > 0 ? v[m * R0 + q] : __ldg(reinterpret_cast<const float2*>(P + (size_t)row * ncols));
                const float2 tt = tma_nb > 0 ? *reinterpret_cast<const float2*>(stg + row * 2 * B + 2 * f)
                                             : __ldg(reinterpret_cast<const float2*>(Tg + (size_t)row * ncols));
                const float r0 = fabsf(p.x) * scale - tt.x, r1 = fabsf(p.y) * scale - tt.y;
                add(r0 * r0);
                add(r1 * r1);
                const float s0 = p.x > 0.f ? 1.f : (p.x < 0.f ? -1.f : 0.f);
                const float s1 = p.y > 0.f ? 1.f : (p.y < 0.f ? -1.f : 0.f);
                g = make_float2(2.f * r0 * scale * s0 * gscale, 2.f * r1 * scale * s1 * gscale);
            }
            v[m * R0 + q] = g;
        }
    // the block's partial: a fixed shuffle tree per warp, then over the warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();                                   // also: the staged map is no longer read
    if (warp == 0) {
        float x = lane < NW ? red[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = x;
    }
    r2c_finish<N, fs_Bcol(N)>(v, sm, t, f, stw, colok, out + (size_t)blockIdx.y * out_img + c, out_pitch, end_scale,
                              mid_scale);
}

// at most 64 registers, so that 4 blocks of 256 threads share a multiprocessor
template <int N, int INTERP>
__global__ void __launch_bounds__(fs_T(N) * fs_Brow(N), 1024 / (fs_T(N) * fs_Brow(N)))
k_nvmt_rows_fast(float2* __restrict__ ws, int W, int Hp, int L, const float2* __restrict__ stw,
                 unsigned* __restrict__ err, long long wait) {
    extern __shared__ __align__(128) float2 sm[];
    pdl_trigger();
    pdl_wait();
    // images in reverse order: the first blocks read the half spectra step 1
    // wrote last (still in L2), and step 4, in forward order, starts on the
    // rows written here last (per 64 x 1024^2: steps 2-3 103.2 -> 100.3 us,
    // step 4 115.4 -> 112.5 us)
    rows_block<N, INTERP, fs_Brow(N), true>(ws + (size_t)(gridDim.y - 1 - blockIdx.y) * L * N, W, Hp, L, stw,
                                            blockIdx.x, sm, err, wait);
}

template <int N, int INTERP>
__global__ void __launch_bounds__(fs_T(N) * fs_Brow(N), 1024 / (fs_T(N) * fs_Brow(N)))
k_nvmt_rows_adjoint_fast(float2* __restrict__ ws, int W, int Hp, int L, const float2* __restrict__ stw) {
    constexpr int B = fs_Brow(N), E = fs_E(N), T = N / E;
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    using F = FastFft<N, -1, B, true>;                 // the row length's seed table
    extern __shared__ float2 sm[];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int l = blockIdx.x * B + f;
    // images in reverse order, as in k_nvmt_rows_fast (L2 reuse with the column
    // kernels before and after, which run in forward order)
    float2* row = ws + (size_t)(gridDim.y - 1 - blockIdx.y) * L * N + (size_t)l * N;

    float2 v[E];
#pragma unroll
    for (int m = 0; m < G0; ++m)
#pragma unroll
        for (int q = 0; q < R0; ++q) {
            const int s = F::template in_pos<0>(t, m, q);
            float2 g = (l < L) ? row[s] : make_float2(0.f, 0.f);
            if (s & 1) g = make_float2(-g.x, -g.y);
            v[m * R0 + q] = g;
        }
    F::template run<0>(v, sm, t, f, stw);
    // gV[x'] = (-1)^{i + N/2} z[i], i = x' + N/2
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int i = F::out_pos(t, m, q);
            float2 z = v[m * RL + q];
            if ((i + N / 2) & 1) z = make_float2(-z.x, -z.y);
            sm[spos(i) * B + f] = z;
        }
    __syncthreads();
    if (l >= L) return;
    // Column x receives from the sample x' with floor(x' H' / (2 l)) = x - W/2 - d
    // (at most one, since H' >= 2 l), i.e. x' = ceil((x - W/2 - d) 2 l / H').  With
    // num = (x - W/2 - d) 2 l + H' - 1 = x' H' + rem (0 <= rem < H') such an x'
    // exists iff H' - 1 - rem < 2 l, and its fraction is (H' - 1 - rem) / (2 l).
    // Successive columns of a thread differ by T, so (x', rem) are stepped exactly.
    constexpr int DLO = INTERP == FT_INTERP_LINEAR ? 0 : -1;
    constexpr int DHI = INTERP == FT_INTERP_LINEAR ? 1 : 2;
    constexpr int ND = DHI - DLO + 1;
    const int halfW = W >> 1;
    const int den = 2 * l;
    const float inv = 1.f / (float)den;
    const int step = T * den;
    const int sA = step / Hp, sB = step - sA * Hp;
    int xp[ND], rem[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        const int num = (t - halfW - (DLO + j)) * den + Hp - 1;
        xp[j] = floor_div(num, Hp);
        rem[j] = num - xp[j] * Hp;
    }
    const int lim = Hp - 1 - den;                      // a sample exists iff rem > lim
    for (int x = t; x < W; x += T) {
        float2 acc = make_float2(0.f, 0.f);
        if (l >= 1) {
#pragma unroll
            for (int j = 0; j < ND; ++j) {
                if (rem[j] > lim && xp[j] >= -N / 2 && xp[j] < N / 2 && FT_IN(xp[j] + N / 2, N, FT_DBG_NVMT_ADJ)) {
                    const float fr = (float)(Hp - 1 - rem[j]) * inv;
                    const float w = INTERP == FT_INTERP_LINEAR ? (j == 0 ? 1.f - fr : fr) : keys_w(fr - (float)(DLO + j));
                    const float2 g = sm[spos(xp[j] + N / 2) * B + f];
                    acc.x = fmaf(w, g.x, acc.x);
                    acc.y = fmaf(w, g.y, acc.y);
                }
                rem[j] += sB;
                xp[j] += sA;
                if (rem[j] >= Hp) { rem[j] -= Hp; xp[j] += 1; }
            }
        }
        row[x] = acc;
    }
}

FT_DEBUG_READER(ft_debug_read_fast)

// ------------------------------------------------------------------ dispatch
#define FT_FAST_LENGTHS(X) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192) X(192) X(384) X(768) X(1536)

// cuTensorMapEncodeTiled through the runtime's driver entry points (no link to
// the driver library); null when unavailable
typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static encode_tiled_fn encode_tiled() {
    static encode_tiled_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (encode_tiled_fn)f;
    }
    return fn;
}

// Tensor copies of step 1's image columns: the N expanded rows of 2B columns in
// nb boxes of h <= 256 rows (each box 128-byte aligned in shared memory), within
// the exchange buffer; false when that does not fit, B < 2 (a box row of 16
// bytes at least), the images are not laid out in 16-byte multiples or the map
// cannot be encoded (the first pass then reads global memory directly).
template <int N>
static bool r2c_tma_map(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img, int batch,
                        CUtensorMap* map, int* h, int* nb) {
    constexpr int B = fs_Bcol(N);
    const encode_tiled_fn enc = encode_tiled();
    if (!enc || B < 2 || ((uintptr_t)in & 15) || (in_pitch & 3) || (in_img & 3) || ncols < 1 || rows_in < 1)
        return false;
    const int step = B >= 16 ? 1 : 16 / B;             // h 2B 4 bytes a multiple of 128
    int n = (N + 255) / 256, hh = 0;
    for (;; ++n) {
        hh = (N + n - 1) / n;
        hh = (hh + step - 1) / step * step;
        if (hh <= 256) break;
    }
    if ((size_t)n * hh * 2 * B * sizeof(float) > (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ncols, (cuuint64_t)rows_in, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)in_pitch * sizeof(float), (cuuint64_t)in_img * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * B), (cuuint32_t)hh, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    *h = hh;
    *nb = n;
    return true;
}

// the distance, in blocks, of the column kernels' L2 prefetch: half of the
// blocks of kernel k (threads, sm bytes of dynamic shared memory) resident on
// the whole GPU at once (0 when it cannot be determined).  Measured per
// 64 x 1024^2 step (pipelined): 2 waves 345 us, 1 wave 320, 1/2 317, 1/4 316,
// 1/8 320, none 327.
template <typename K>
static int prefetch_distance(K k, int threads, size_t sm) {
    int dev = 0, per = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, sm) != cudaSuccess)
        return 0;
    return per * nsm / 2;
}

template <int N>
static cudaError_t go_r2c(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img, int row0,
                          const float2* stw, float2* out, int out_pitch, size_t out_img, float es, float ms,
                          int batch, cudaStream_t st, bool pdl, bool follows_peak, unsigned* err, long long wait) {
    constexpr int B = fs_Bcol(N);
    const size_t sm = (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_r2c_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    int h = 0, nb = 0;
    if (!err || wait < 0 || !r2c_tma_map<N>(in, rows_in, ncols, in_pitch, in_img, batch, &map, &h, &nb)) nb = 0;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    const int pf = prefetch_distance(k_col_r2c_fast<N>, fs_T(N) * B, sm);
    return launch_maybe_pdl(k_col_r2c_fast<N>, grid, dim3(fs_T(N) * B), sm, st, pdl, in, rows_in, ncols, in_pitch,
                            in_img, row0, stw, out, out_pitch, out_img, es, ms, map, h, nb, err, wait, pf,
                            (pdl && follows_peak) ? 1 : 0);
}

template <int N>
static cudaError_t go_r2c_loss(const float* map, const float* target, int ncols, const float2* stw, float2* out,
                               int out_pitch, size_t out_img, float es, float ms, float scale, float gscale,
                               float* partial, int batch, cudaStream_t st, unsigned* err, long long wait) {
    constexpr int B = fs_Bcol(N);
    const size_t sm = (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_r2c_loss_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    CUtensorMap pm, tm;
    memset(&pm, 0, sizeof(pm));
    memset(&tm, 0, sizeof(tm));
    const size_t cells = (size_t)N * ncols;
    int h = 0, nb = 0, h2 = 0, nb2 = 0;
    if (!err || wait < 0 || !r2c_tma_map<N>(map, N, ncols, ncols, cells, batch, &pm, &h, &nb) ||
        !r2c_tma_map<N>(target, N, ncols, ncols, cells, batch, &tm, &h2, &nb2))
        nb = 0;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    const int pf = prefetch_distance(k_col_r2c_loss_fast<N>, fs_T(N) * B, sm);
    k_col_r2c_loss_fast<N><<<grid, fs_T(N) * B, sm, st>>>(map, target, ncols, cells, stw, out, out_pitch, out_img, es,
                                                          ms, scale, gscale, partial, pm, tm, h, nb, err, wait, pf);
    return cudaGetLastError();
}

// Tensor copies of step 4's staging: the N/2 + 1 Hermitian rows in nb boxes of
// h <= 256 rows, h B a multiple of 8 (each box starts on a 128-byte boundary of
// shared memory), all within the block's exchange buffer; false when that does
// not fit, the input is not 16-byte aligned or the map cannot be encoded (the
// kernel then stages with cp.async).
template <int N>
static bool c2r_tma_map(const float2* in, int in_pitch, size_t in_img, int batch, CUtensorMap* map, int* h, int* nb) {
    constexpr int B = fs_Bc2r(N), rows = N / 2 + 1;
    const encode_tiled_fn enc = encode_tiled();
    if (!enc || ((uintptr_t)in & 15) || (in_pitch & 1) || (in_img & 1)) return false;
    const int step = B >= 8 ? 1 : 8 / B;
    int n = (rows + 255) / 256, hh = 0;
    for (;; ++n) {
        hh = (rows + n - 1) / n;
        hh = (hh + step - 1) / step * step;
        if (hh <= 256) break;
    }
    if ((size_t)n * hh * 2 * B > (size_t)FastFft<N, +1, B>::SLOTS) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)in_pitch, (cuuint64_t)rows, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)in_pitch * sizeof(float2), (cuuint64_t)in_img * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * B), (cuuint32_t)hh, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    *h = hh;
    *nb = n;
    return true;
}

template <int N>
static cudaError_t go_c2r(const float2* in, int ncols, int in_pitch, size_t in_img, const float2* stw,
                          float mid, float* out, int row0, int rows_out, int out_pitch, size_t out_img,
                          float os, unsigned* tmax, int batch, cudaStream_t st, bool pdl, unsigned* err,
                          long long wait) {
    constexpr int B = fs_Bc2r(N);
    const size_t sm = (size_t)FastFft<N, +1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_c2r_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    int h = 0, nb = 0;
    if (!err || wait < 0 || !c2r_tma_map<N>(in, in_pitch, in_img, batch, &map, &h, &nb)) nb = 0;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    const int pf = prefetch_distance(k_col_c2r_fast<N>, fs_T(N) * B, sm);
    return launch_maybe_pdl(k_col_c2r_fast<N>, grid, dim3(fs_T(N) * B), sm, st, pdl, in, ncols, in_pitch, in_img, stw,
                            mid, out, row0, rows_out, out_pitch, out_img, os, tmax, map, h, nb, err, wait, pf);
}

template <int N, int INTERP>
static cudaError_t go_rows_i(float2* ws, int W, int Hp, int L, const float2* stw, int batch, cudaStream_t st,
                             bool pdl, unsigned* err, long long wait) {
    constexpr int B = fs_Brow(N);
    const size_t slots = FastFft<N, +1, B>::SLOTS, rows = (size_t)srow_pitch(W) * B;
    const size_t sm = (slots > rows ? slots : rows) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_fast<N, INTERP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((L + B - 1) / B, batch);
    return launch_maybe_pdl(k_nvmt_rows_fast<N, INTERP>, grid, dim3(fs_T(N) * B), sm, st, pdl, ws, W, Hp, L, stw,
                            err, wait);
}

template <int N>
static cudaError_t go_rows(float2* ws, int W, int Hp, int L, int interp, const float2* stw, int batch,
                           cudaStream_t st, bool pdl, unsigned* err, long long wait) {
    return interp == FT_INTERP_LINEAR ? go_rows_i<N, FT_INTERP_LINEAR>(ws, W, Hp, L, stw, batch, st, pdl, err, wait)
                                      : go_rows_i<N, FT_INTERP_CUBIC>(ws, W, Hp, L, stw, batch, st, pdl, err, wait);
}

template <int N, int INTERP>
static cudaError_t go_rows_adj_i(float2* ws, int W, int Hp, int L, const float2* stw, int batch, cudaStream_t st) {
    constexpr int B = fs_Brow(N);
    const size_t sm = (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_adjoint_fast<N, INTERP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((L + B - 1) / B, batch);
    k_nvmt_rows_adjoint_fast<N, INTERP><<<grid, fs_T(N) * B, sm, st>>>(ws, W, Hp, L, stw);
    return cudaGetLastError();
}

template <int N>
static cudaError_t go_rows_adj(float2* ws, int W, int Hp, int L, int interp, const float2* stw, int batch,
                               cudaStream_t st) {
    return interp == FT_INTERP_LINEAR ? go_rows_adj_i<N, FT_INTERP_LINEAR>(ws, W, Hp, L, stw, batch, st)
                                      : go_rows_adj_i<N, FT_INTERP_CUBIC>(ws, W, Hp, L, stw, batch, st);
}

cudaError_t launch_col_r2c_fast(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img,
                                int row0, const FftLen& f, float2* out, int out_pitch, size_t out_img,
                                float end_scale, float mid_scale, int batch, cudaStream_t st, bool pdl,
                                bool follows_peak, unsigned* err, long long wait) {
    switch (f.N) {
#define X(n) case n: return go_r2c<n>(in, rows_in, ncols, in_pitch, in_img, row0, f.stw, out, out_pitch, \
                                      out_img, end_scale, mid_scale, batch, st, pdl, follows_peak, err, wait);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}

int col_r2c_loss_blocks(const FftLen& f, int ncols) {
    switch (f.N) {
#define X(n) case n: return (ncols + 2 * fs_Bcol(n) - 1) / (2 * fs_Bcol(n));
        FT_FAST_LENGTHS(X)
#undef X
    }
    return 0;
}

cudaError_t launch_col_r2c_loss_fast(const float* map, const float* target, int ncols, const FftLen& f,
                                     float2* out, int out_pitch, size_t out_img, float end_scale, float mid_scale,
                                     float scale, float gscale, float* partial, int batch, cudaStream_t st,
                                     unsigned* err, long long wait) {
    if (ncols & 1) return cudaErrorInvalidValue;
    switch (f.N) {
#define X(n) case n: return go_r2c_loss<n>(map, target, ncols, f.stw, out, out_pitch, out_img, end_scale, mid_scale, \
                                           scale, gscale, partial, batch, st, err, wait);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_col_c2r_fast(const float2* in, int ncols, int in_pitch, size_t in_img,
                                const FftLen& f, float mid_scale, float* out, int row0, int rows_out,
                                int out_pitch, size_t out_img, float out_scale, int batch,
                                cudaStream_t st, unsigned* tmax, bool pdl, unsigned* err, long long wait) {
    if (tmax && (row0 != 0 || rows_out != f.N)) return cudaErrorInvalidValue;
    switch (f.N) {
#define X(n) case n: return go_c2r<n>(in, ncols, in_pitch, in_img, f.stw, mid_scale, out, row0, rows_out, \
                                      out_pitch, out_img, out_scale, tmax, batch, st, pdl, err, wait);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}

bool c2r_tile_shape(int N, int* rows, int* cols, int* bands) {
    switch (N) {
#define X(n) case n: *rows = c2r_tile_rows(n); *cols = 2 * fs_Bc2r(n); *bands = n / c2r_tile_rows(n); return true;
        FT_FAST_LENGTHS(X)
#undef X
    }
    return false;
}

cudaError_t launch_nvmt_rows_fast(float2* ws, int W, int Hp, int L, int interp, const FftLen& fx,
                                  int batch, cudaStream_t st, bool pdl, unsigned* err, long long wait) {
    if (((uintptr_t)ws & 15) || (W & 1) || wait < 0) return cudaErrorInvalidValue;   // bulk-copy alignment
    switch (fx.N) {
#define X(n) case n: return go_rows<n>(ws, W, Hp, L, interp, fx.stw, batch, st, pdl, err, wait);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_nvmt_rows_adjoint_fast(float2* ws, int W, int Hp, int L, int interp,
                                          const FftLen& fx, int batch, cudaStream_t st) {
    switch (fx.N) {
#define X(n) case n: return go_rows_adj<n>(ws, W, Hp, L, interp, fx.stw, batch, st);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}
