// Discrete Fourier transforms as tensor-core GEMMs (the split-precision variant
// of the FFT stages).
//
// A batch of length-64 complex DFTs y[v][k] = sum_n x[v][n] exp(sign 2 pi i k n / 64)
// is one real GEMM per 64 vectors:
//     D (128 x 64) = A (128 x 128) * B^T,   A = [[Fr, -Fi], [Fi, Fr]],
//     B row v = [Re x[v][0..63], Im x[v][0..63]],   D = [Re y ; Im y] (rows k, k + 64)
// with F[k][n] = exp(sign 2 pi i k n / 64).  Both operands are split into a high
// and a low 16-bit part (BF16 or FP16) of the FP32 values and
//     D = Ahi Bhi + Ahi Blo + Alo Bhi
// is accumulated in FP32 in tensor memory by tcgen05.mma (M = 128, N = 64,
// K = 16 per instruction, 24 instructions).  The inputs are scaled by a power of
// two so that FP16 stays in range; the scale is undone on output.
//
// k_tc_dft64 is the building block and its own check (ft_tc_dft64); the row
// transform of length 4096 = 64 x 64 in k_tc_rows4096 composes two of these GEMMs
// with a twiddle pass in between (four-step FFT).
#include "tc_common.cuh"

#define TC_THREADS 128
#define TC_A_BYTES (128 * 128 * 2)
#define TC_B_BYTES (64 * 128 * 2)

// e^{+2 pi i t / 64}, t = 0..63 (FP64 values rounded to FP32, set once per device)
static __device__ float2 g_w64[64];

// Fill A (hi, lo) for exp(sign 2 pi i k n / 64) in the K-major layout.
template <int FMT>
__device__ void build_dft_matrix(unsigned char* a_hi, unsigned char* a_lo, const float2* w, int sign) {
    for (int idx = threadIdx.x; idx < 128 * 128; idx += blockDim.x) {
        const int r = idx >> 7, c = idx & 127;
        const int k = r & 63, n = c & 63;
        const float2 e = w[(k * n) & 63];
        const float fr = e.x, fi = sign > 0 ? e.y : -e.y;
        float v;
        if (r < 64) v = c < 64 ? fr : -fi;
        else v = c < 64 ? fi : fr;
        uint16_t hi, lo;
        split16<FMT>(v, hi, lo);
        const uint32_t off = kmajor_off(r, c, 128);
        *reinterpret_cast<uint16_t*>(a_hi + off) = hi;
        *reinterpret_cast<uint16_t*>(a_lo + off) = lo;
    }
}

// 3 x 8 MMAs D = Ahi Bhi + Ahi Blo + Alo Bhi, then commit to mbar
template <int FMT>
__device__ __forceinline__ void issue_split_gemm(uint32_t tmem_d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                                 uint32_t b_lo, uint32_t mbar) {
    constexpr uint32_t idesc = idesc_f16(FMT, 128, 64);
    const uint32_t as[3] = {a_hi, a_hi, a_lo};
    const uint32_t bs[3] = {b_hi, b_lo, b_hi};
#pragma unroll
    for (int term = 0; term < 3; ++term)
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
            tc_mma(tmem_d, smem_desc(as[term] + ks * 256, 128, 2048), smem_desc(bs[term] + ks * 256, 128, 2048),
                   idesc, (term | ks) != 0);
    tc_commit(mbar);
}

template <int FMT>
__global__ void __launch_bounds__(TC_THREADS)
k_tc_dft64(const float2* __restrict__ x, float2* __restrict__ y, int nvec, int sign, unsigned* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* a_hi = sm;
    unsigned char* a_lo = a_hi + TC_A_BYTES;
    unsigned char* b_hi = a_lo + TC_A_BYTES;
    unsigned char* b_lo = b_hi + TC_B_BYTES;
    float* stage = reinterpret_cast<float*>(b_lo + TC_B_BYTES);     // [64 vectors][64][2]
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float red[TC_THREADS];
    const int v0 = blockIdx.x * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    build_dft_matrix<FMT>(a_hi, a_lo, g_w64, sign);
    // a power-of-two scale that brings max |x| near 2^10
    float mx = 0.f;
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int v = v0 + (i >> 6);
        if (v < nvec) {
            const float2 t = x[(size_t)v * 64 + (i & 63)];
            mx = fmaxf(mx, fmaxf(fabsf(t.x), fabsf(t.y)));
        }
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = TC_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const int e = red[0] > 0.f ? ilogbf(red[0]) : 0;
    const float scale = ldexpf(1.f, 10 - e), unscale = ldexpf(1.f, e - 10);
    for (int i = threadIdx.x; i < 64 * 128; i += blockDim.x) {
        const int vl = i >> 7, c = i & 127;
        const int v = v0 + vl;
        float val = 0.f;
        if (v < nvec) {
            const float2 t = x[(size_t)v * 64 + (c & 63)];
            val = (c < 64 ? t.x : t.y) * scale;
        }
        uint16_t hi, lo;
        split16<FMT>(val, hi, lo);
        const uint32_t off = kmajor_off(vl, c, 128);
        *reinterpret_cast<uint16_t*>(b_hi + off) = hi;
        *reinterpret_cast<uint16_t*>(b_lo + off) = lo;
    }
    fence_async_smem();
    if (threadIdx.x == 0) mbar_init(smem_u32(&mbar), 1);
    if (warp == 0) {
        tc_alloc(smem_u32(&tmem_base), 64);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (threadIdx.x == 0)
        issue_split_gemm<FMT>(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_hi), smem_u32(b_lo), smem_u32(&mbar));
    bool ok = mbar_wait(smem_u32(&mbar), 0);
    if (!ok) {
        atomicOr(err, 1u);
        ok = mbar_wait(smem_u32(&mbar), 0);            // let our own MMAs drain before freeing TMEM
    }
    tc_fence_after();
    // row r = 32 warp + lane of D: Re (r < 64) or Im (r >= 64) of y[v0 + col][r & 63]
    const int r = 32 * warp + lane;
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
        float d[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * c16, d);
#pragma unroll
        for (int j = 0; j < 16; ++j) stage[((16 * c16 + j) * 64 + (r & 63)) * 2 + (r >> 6)] = ok ? d[j] * unscale : __int_as_float(0x7fc00000);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 64);
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int v = v0 + (i >> 6);
        if (v < nvec) y[(size_t)v * 64 + (i & 63)] = make_float2(stage[2 * i], stage[2 * i + 1]);
    }
}

static size_t dft64_smem() { return 2 * TC_A_BYTES + 2 * TC_B_BYTES + 64 * 64 * 2 * sizeof(float); }

// e^{+2 pi i t / 64} in FP64, rounded once
static cudaError_t set_w64() {
    float2 w[64];
    for (int t = 0; t < 64; ++t) {
        const double th = 6.283185307179586476925286766559 * t / 64.0;
        w[t] = make_float2((float)cos(th), (float)sin(th));
    }
    return cudaMemcpyToSymbol(g_w64, w, sizeof(w));
}

cudaError_t launch_tc_dft64(const float2* x, float2* y, int nvec, int sign, int fmt, unsigned* err,
                            cudaStream_t st) {
    static int ready[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !ready[dev]) {
        if ((e = set_w64()) != cudaSuccess) return e;
        ready[dev] = 1;
    }
    const size_t sm = dft64_smem();
    const dim3 grid((nvec + 63) / 64);
    if (fmt == 1) {
        if ((e = cudaFuncSetAttribute(k_tc_dft64<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        k_tc_dft64<1><<<grid, TC_THREADS, sm, st>>>(x, y, nvec, sign, err);
    } else {
        if ((e = cudaFuncSetAttribute(k_tc_dft64<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        k_tc_dft64<0><<<grid, TC_THREADS, sm, st>>>(x, y, nvec, sign, err);
    }
    return cudaGetLastError();
}
