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
// transform of length 4096 = 64 x 64 in k_nvmt_rows_tc4096 composes two of these GEMMs
// with a twiddle pass in between (four-step FFT).
#include "fft_fast.cuh"
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

// g_w64 is set once per device (the first call on a device does it)
static cudaError_t ensure_w64() {
    static int ready[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!ready[dev]) {
        if ((e = set_w64()) != cudaSuccess) return e;
        ready[dev] = 1;
    }
    return cudaSuccess;
}

cudaError_t tc_prepare() { return ensure_w64(); }

cudaError_t launch_tc_dft64(const float2* x, float2* y, int nvec, int sign, int fmt, unsigned* err,
                            cudaStream_t st) {
    cudaError_t e = ensure_w64();
    if (e != cudaSuccess) return e;
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

// ---------------------------------------------------------------------------
// Steps 2-3 for n_slope = 4096 with the step-3 transform on the tensor cores.
// Per frequency row: the NVMT gather (as in the FP32 row kernels) of
// V[n] (-1)^n, then the four-step DFT with 4096 = 64 x 64 (n = n1 + 64 n2,
// k = k2 + 64 k1), sign +1:
//     A[k2][n1]  = sum_n2 exp(+2 pi i n2 k2 / 64) V[n1 + 64 n2]     GEMM 1 (B row n1)
//     A'[k2][n1] = A[k2][n1] exp(+2 pi i n1 k2 / 4096)                 FP32 twiddles
//     Y[k1][k2]  = sum_n1 exp(+2 pi i n1 k1 / 64) A'[k2][n1]           GEMM 2 (B row k2)
//     G[k2 + 64 k1] = Y[k1][k2] (-1)^{k + S/2}
// The gather writes GEMM 1's operand directly (each thread builds 16-byte runs
// of 8 columns of one operand row), the twiddle pass writes GEMM 2's.  Each
// operand gets a power-of-two scale, undone on output: for GEMM 1 from a bound
// on |V| (the largest component of the spectrum row times the interpolator's
// sum of |weights|), for GEMM 2 from the largest component of A (the twiddle
// keeps |A'| = |A| <= sqrt(2) max component).
//
// Persistent blocks of two independent row groups (4 warps each) that share the
// DFT matrix in shared memory: each group has its own operand buffers, staging
// area, 64 TMEM columns, mbarrier and named barrier, so one group's SIMT work
// (gather, twiddles, stores) overlaps the other's tensor-core GEMMs.
#define TCR_GROUPS 2
#define TCR_GT 128                                     // threads per group
#define TCR_THREADS (TCR_GROUPS * TCR_GT)
#define TCR_S 4096
#define TCR_PITCH 65                                   // stage row pitch (floats): conflict-free rows and columns

static constexpr size_t tcr_stage_bytes(int W) {
    return (size_t)128 * TCR_PITCH * 4 > (size_t)(W + 2) * 8 ? (size_t)128 * TCR_PITCH * 4 : (size_t)(W + 2) * 8;
}
static size_t tcr_group_bytes(int W) { return ((2 * TC_B_BYTES + tcr_stage_bytes(W)) + 1023) & ~(size_t)1023; }
static size_t tcr_smem(int W) { return 2 * TC_A_BYTES + TCR_GROUPS * tcr_group_bytes(W); }

__device__ __forceinline__ void group_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(TCR_GT) : "memory");
}
// named-barrier sync of the group that also ORs v over its threads
__device__ __forceinline__ bool group_sync_or(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(TCR_GT)
        : "memory");
    return r != 0;
}

template <int FMT>
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
    uint16_t h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split16<FMT>(x[j], h[j], l[j]);
    hi = make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16), h[4] | ((uint32_t)h[5] << 16),
                    h[6] | ((uint32_t)h[7] << 16));
    lo = make_uint4(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16), l[4] | ((uint32_t)l[5] << 16),
                    l[6] | ((uint32_t)l[7] << 16));
}

// Write 8 complex values (columns c0..c0+7 of operand row r) as hi/lo: real parts
// to columns c0.., imaginary parts to c0 + 64.. of the K = 128 K-major tile.
template <int FMT>
__device__ __forceinline__ void put8(unsigned char* b_hi, unsigned char* b_lo, int r, int kg, const float (&re)[8],
                                     const float (&im)[8]) {
    const uint32_t off = (uint32_t)(((r >> 3) * 16 + kg) * 128 + (r & 7) * 16);
    uint4 h, l;
    split8<FMT>(re, h, l);
    *reinterpret_cast<uint4*>(b_hi + off) = h;
    *reinterpret_cast<uint4*>(b_lo + off) = l;
    split8<FMT>(im, h, l);
    *reinterpret_cast<uint4*>(b_hi + off + 1024) = h;
    *reinterpret_cast<uint4*>(b_lo + off + 1024) = l;
}

template <int FMT, int INTERP>
__global__ void __launch_bounds__(TCR_THREADS, 1)
k_nvmt_rows_tc4096(float2* __restrict__ ws, int W, int Hp, int L, int total_rows, size_t group_bytes,
                   const float2* __restrict__ tw, unsigned* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int S = TCR_S, T = TCR_GT;
    const int g = threadIdx.x / TCR_GT, gt = threadIdx.x % TCR_GT;   // group, thread in group
    const int warp = gt >> 5, lane = gt & 31;          // warp in group = TMEM lane quarter
    unsigned char* a_hi = sm;
    unsigned char* a_lo = a_hi + TC_A_BYTES;
    unsigned char* b_hi = a_lo + TC_A_BYTES + g * group_bytes;
    unsigned char* b_lo = b_hi + TC_B_BYTES;
    float* stage = reinterpret_cast<float*>(b_lo + TC_B_BYTES);         // [128][TCR_PITCH] accumulator copy
    float2* srow = reinterpret_cast<float2*>(stage);                     // the spectrum row (aliases stage)
    __shared__ uint64_t mbar[TCR_GROUPS];
    __shared__ uint32_t tmem_base;
    __shared__ float red[TCR_GROUPS][4];
    const int bar = 1 + g;                              // named barrier of the group

    build_dft_matrix<FMT>(a_hi, a_lo, g_w64, +1);
    if (threadIdx.x == 0)
        for (int j = 0; j < TCR_GROUPS; ++j) mbar_init(smem_u32(&mbar[j]), 1);
    if (threadIdx.x < 32) {
        tc_alloc(smem_u32(&tmem_base), 64 * TCR_GROUPS);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base + 64 * g;          // this group's 64 accumulator columns
    const uint32_t mb = smem_u32(&mbar[g]);
    uint32_t parity = 0;

    auto group_max = [&](float v) -> float {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[g][warp] = v;
        group_sync(bar);
        const float r = fmaxf(fmaxf(red[g][0], red[g][1]), fmaxf(red[g][2], red[g][3]));
        group_sync(bar);
        return r;
    };
    // issue the split GEMM on the group's B and wait; group-uniform result
    auto gemm = [&]() -> bool {
        fence_async_smem();
        group_sync(bar);
        tc_fence_after();
        if (gt == 0)
            issue_split_gemm<FMT>(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_hi), smem_u32(b_lo), mb);
        bool ok = mbar_wait(mb, parity);
        if (!ok) {
            atomicOr(err, 1u);
            mbar_wait(mb, parity);                      // let our own MMAs drain
        }
        parity ^= 1u;
        tc_fence_after();
        return !group_sync_or(bar, !ok);
    };
    // accumulator rows 32 warp + lane, all 64 columns -> stage; returns the max |value|
    auto read_d = [&]() -> float {
        float mx = 0.f;
        const int r = 32 * warp + lane;
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
            float d[16];
            tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * c16, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                stage[r * TCR_PITCH + 16 * c16 + j] = d[j];
                mx = fmaxf(mx, fabsf(d[j]));
            }
        }
        tc_fence_before();
        return mx;
    };

    for (int job = blockIdx.x * TCR_GROUPS + g; job < total_rows; job += gridDim.x * TCR_GROUPS) {
        const int l = job % L;
        float2* row = ws + (size_t)job * S;            // row l of image job / L
        if (l == 0) {                                   // the DC row is zero
            for (int k = gt; k < S; k += T) row[k] = make_float2(0.f, 0.f);
            continue;
        }
        for (int i = gt; i < W / 2; i += T) cp_async16(srow + 2 * i, row + 2 * i);
        cp_async_wait_all();
        float mx = 0.f;
        for (int i = gt; i < W / 2; i += T) {           // this thread's own copies
            const float4 v = *reinterpret_cast<const float4*>(srow + 2 * i);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        mx = group_max(mx) * (INTERP == FT_INTERP_LINEAR ? 1.f : 1.25f);   // sum of |Keys weights| <= 1.25
        const int e1 = mx > 0.f ? ilogbf(mx) : 0;
        const float s1 = ldexpf(1.f, 10 - e1);
        // gather V[n1 + 64 n2] for n2 = 8 kg .. 8 kg + 7 straight into B row n1
        {
            const int den = 2 * l;
            const float inv = 1.f / (float)den;
            const int step = 64 * Hp;                   // n advances by 64 per n2
            const int sA = step / den, sB = step - sA * den;
            const int halfW = W >> 1;
            const float2 zero = make_float2(0.f, 0.f);
            for (int item = gt; item < 512; item += T) {
                const int r = (item & 7) | ((item >> 6) << 3), kg = (item >> 3) & 7;
                const int n0 = r + 512 * kg;
                const int num = (n0 - S / 2) * Hp;
                int qf = floor_div(num, den), rem = num - qf * den;
                float re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float fr = (float)rem * inv;
                    const int cc = qf + halfW;
                    float2 acc;
                    if (INTERP == FT_INTERP_LINEAR) {
                        const float2 a0 = (unsigned)cc < (unsigned)W ? srow[cc] : zero;
                        const float2 a1 = (unsigned)(cc + 1) < (unsigned)W ? srow[cc + 1] : zero;
                        acc = make_float2(fmaf(fr, a1.x - a0.x, a0.x), fmaf(fr, a1.y - a0.y, a0.y));
                    } else {
                        acc = zero;
#pragma unroll
                        for (int d = -1; d <= 2; ++d) {
                            const float2 a = (unsigned)(cc + d) < (unsigned)W ? srow[cc + d] : zero;
                            const float w = keys_w(fr - (float)d);
                            acc.x = fmaf(w, a.x, acc.x);
                            acc.y = fmaf(w, a.y, acc.y);
                        }
                    }
                    const float sg = (r & 1) ? -s1 : s1;          // (-1)^n, n = r + 64 (8 kg + j)
                    re[j] = acc.x * sg;
                    im[j] = acc.y * sg;
                    rem += sB;
                    qf += sA;
                    if (rem >= den) { rem -= den; qf += 1; }
                }
                put8<FMT>(b_hi, b_lo, r, kg, re, im);
            }
        }
        if (!gemm()) break;
        mx = group_max(read_d());                       // also orders the stage writes before the reads below
        const int e2 = mx > 0.f ? ilogbf(mx) : 0;
        const float s2 = ldexpf(1.f, 10 - e2);
        // twiddle A[k2][n1] (rows k2 / k2 + 64 of stage) and write B row k2
        for (int item = gt; item < 512; item += T) {
            const int k2 = (item & 7) | ((item >> 6) << 3), kg = (item >> 3) & 7;
            float re[8], im[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n1 = 8 * kg + j;
                const float2 w = __ldg(tw + n1 * k2);   // exp(-2 pi i n1 k2 / S), n1 k2 < S
                const float a = stage[k2 * TCR_PITCH + n1], b = stage[(k2 + 64) * TCR_PITCH + n1];
                re[j] = (a * w.x + b * w.y) * s2;       // (a + i b) conj(w)
                im[j] = (b * w.x - a * w.y) * s2;
            }
            put8<FMT>(b_hi, b_lo, k2, kg, re, im);
        }
        if (!gemm()) break;
        read_d();
        group_sync(bar);
        const float un = ldexpf(1.f, e1 + e2 - 20);
        for (int k = gt; k < S; k += T) {
            const int k1 = k >> 6, k2 = k & 63;
            const float sg = ((k + S / 2) & 1) ? -un : un;
            row[k] = make_float2(stage[k1 * TCR_PITCH + k2] * sg, stage[(k1 + 64) * TCR_PITCH + k2] * sg);
        }
        group_sync(bar);                                // stage is the next row's srow
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc_dealloc(tmem_base, 64 * TCR_GROUPS);
}

template <int FMT, int INTERP>
static cudaError_t go_tc_rows(float2* ws, int W, int Hp, int L, int batch, const float2* tw, unsigned* err,
                              cudaStream_t st) {
    const size_t sm = tcr_smem(W);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_tc4096<FMT, INTERP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int total = batch * L;
    const int blocks = (total + TCR_GROUPS - 1) / TCR_GROUPS;
    k_nvmt_rows_tc4096<FMT, INTERP><<<blocks < sms ? blocks : sms, TCR_THREADS, sm, st>>>(
        ws, W, Hp, L, total, tcr_group_bytes(W), tw, err);
    return cudaGetLastError();
}

cudaError_t launch_nvmt_rows_tc4096(float2* ws, int W, int Hp, int L, int interp, int fmt, const float2* tw,
                                    unsigned* err, int batch, cudaStream_t st) {
    if (W <= 0 || W > TCR_S || (W & 1)) return cudaErrorInvalidValue;
    cudaError_t e = ensure_w64();
    if (e != cudaSuccess) return e;
    if (interp == FT_INTERP_LINEAR)
        return fmt == 1 ? go_tc_rows<1, FT_INTERP_LINEAR>(ws, W, Hp, L, batch, tw, err, st)
                        : go_tc_rows<0, FT_INTERP_LINEAR>(ws, W, Hp, L, batch, tw, err, st);
    return fmt == 1 ? go_tc_rows<1, FT_INTERP_CUBIC>(ws, W, Hp, L, batch, tw, err, st)
                    : go_tc_rows<0, FT_INTERP_CUBIC>(ws, W, Hp, L, batch, tw, err, st);
}
