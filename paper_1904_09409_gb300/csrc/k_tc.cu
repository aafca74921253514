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

// e^{+2 pi i t / 64} and e^{+2 pi i t / 4096}, t = 0..63 (FP64 values rounded
// to FP32, set once per device)
static __device__ float2 g_w64[64];
static __device__ float2 g_w4096[64];

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

// e^{+2 pi i t / 64} and e^{+2 pi i t / 4096} in FP64, rounded once
static cudaError_t set_w64() {
    float2 w[64], v[64];
    for (int t = 0; t < 64; ++t) {
        const double th = 6.283185307179586476925286766559 * t / 64.0;
        w[t] = make_float2((float)cos(th), (float)sin(th));
        const double ph = 6.283185307179586476925286766559 * t / 4096.0;
        v[t] = make_float2((float)cos(ph), (float)sin(ph));
    }
    cudaError_t e = cudaMemcpyToSymbol(g_w64, w, sizeof(w));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_w4096, v, sizeof(v));
    return e;
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
// A complex 64-point DFT of 64 vectors is two real GEMMs with the same matrix
// [Fr; Fi] (M = 128, K = 64): D1 = [Fr; Fi] Re(B)^T, D2 = [Fr; Fi] Im(B)^T, and
// Re y = Fr Re x - Fi Im x = D1[k] - D2[k + 64], Im y = D2[k] + D1[k + 64],
// combined when the accumulators are read back.  Every operand is split into
// high and low 16-bit parts; D = A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32.
// The gather writes GEMM 1's operands directly (each thread builds 16-byte runs
// of 8 columns of one operand row; the 32 threads of a warp take 32 consecutive
// rows of the same 8 columns, so their reads of consecutive samples and of the
// swizzled stage are conflict-free), the twiddle pass writes GEMM 2's.  Each
// operand gets a power-of-two scale, undone on output: for GEMM 1 from a bound
// on |V| (the largest component of the spectrum row times the interpolator's
// sum of |weights|), for GEMM 2 from the largest component of A (the twiddle
// keeps |A'| = |A| <= sqrt(2) max component).  The twiddle
// exp(+2 pi i t / 4096), t = n1 k2 < 4096, is the product of two 64-entry
// tables (t = 64 a + b) kept in shared memory.
//
// Persistent blocks of three independent row groups (4 warps each) that share
// the DFT matrix in shared memory: each group has its own operand buffers,
// staging area, 128 TMEM columns, mbarrier and named barrier, so the groups'
// SIMT work (gather, twiddles, stores) overlaps their GEMMs.
#define TCR_GT 128                                     // threads per group
#define TCR_MAXG 3                                     // groups per block at most
#define TCR_S 4096
#define TCR_A_BYTES (128 * 64 * 2)                     // [Fr; Fi], K = 64, one 16-bit piece
#define TCR_B_BYTES (64 * 64 * 2)                      // 64 operand rows, K = 64, one piece
#define TCR_STAGE_BYTES (128 * 64 * 4)                 // the accumulator copy (or the staged input)

// Operand format (FMT: 0 FP16, 1 BF16), pieces per FP32 value and row groups
// per block of each precision: FP16 and BF16 hi + lo (3 products), and BF16 in
// three pieces hi + mid + lo (6 products: every pair of order <= 2), which needs
// 1.5 times the operand memory and so runs two groups per block.
template <int PREC>
struct TcPrec {
    static constexpr int FMT = PREC == FT_PRECISION_FP16X3 ? 0 : 1;
    static constexpr int PIECES = PREC == FT_PRECISION_BF16X6 ? 3 : 2;
    static constexpr int GROUPS = PIECES == 3 ? 2 : 3;
    static constexpr int THREADS = GROUPS * TCR_GT;
    static constexpr size_t GROUP_BYTES = (size_t)2 * PIECES * TCR_B_BYTES + TCR_STAGE_BYTES;
    static constexpr size_t SMEM = (size_t)PIECES * TCR_A_BYTES + GROUPS * GROUP_BYTES + 128 * sizeof(float2);
};

// stage element (r, c), r < 128, c < 64: rows of 64 floats, columns XOR-swizzled
// by the row so that row-wise and column-wise warp accesses hit distinct banks
__device__ __forceinline__ int tcr_sw(int r, int c) { return r * 64 + (c ^ (r & 31)); }

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

// x = p[0] + p[1] (+ p[2]) in the operand format, each piece rounded to nearest
// from the remainder of the previous ones
template <int FMT, int PIECES>
__device__ __forceinline__ void split_pieces(float x, uint16_t (&p)[PIECES]) {
    if constexpr (PIECES == 2) {
        split16<FMT>(x, p[0], p[1]);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
        p[0] = __bfloat16_as_ushort(h);
        p[1] = __bfloat16_as_ushort(m);
        p[2] = __bfloat16_as_ushort(l);
    }
}

// Write 8 values (K columns 8 kg .. 8 kg + 7 of operand row r) as 16-bit pieces,
// piece q to the K = 64 K-major tile at dst + q * TCR_B_BYTES (16-byte stores).
template <int FMT, int PIECES>
__device__ __forceinline__ void put8_pieces(unsigned char* dst, uint32_t off, const float (&x)[8]) {
    uint16_t p[8][PIECES];
#pragma unroll
    for (int j = 0; j < 8; ++j) split_pieces<FMT, PIECES>(x[j], p[j]);
#pragma unroll
    for (int q = 0; q < PIECES; ++q)
        *reinterpret_cast<uint4*>(dst + q * TCR_B_BYTES + off) =
            make_uint4(p[0][q] | ((uint32_t)p[1][q] << 16), p[2][q] | ((uint32_t)p[3][q] << 16),
                       p[4][q] | ((uint32_t)p[5][q] << 16), p[6][q] | ((uint32_t)p[7][q] << 16));
}

// 8 complex values of operand row r: real parts to the Re operand, imaginary
// parts to the Im operand (b = [Re pieces | Im pieces], each a K = 64 tile)
template <int FMT, int PIECES>
__device__ __forceinline__ void put8(unsigned char* b, int r, int kg, const float (&re)[8], const float (&im)[8]) {
    const uint32_t off = (uint32_t)(((r >> 3) * 8 + kg) * 128 + (r & 7) * 16);
    put8_pieces<FMT, PIECES>(b, off, re);
    put8_pieces<FMT, PIECES>(b + PIECES * TCR_B_BYTES, off, im);
}

// [Fr; Fi] of exp(SIGN 2 pi i k n / 64) in pieces (piece q at a + q * TCR_A_BYTES), K = 64 K-major
template <int FMT, int PIECES, int SIGN>
__device__ void build_dft_matrix_k64(unsigned char* a) {
    for (int idx = threadIdx.x; idx < 128 * 64; idx += blockDim.x) {
        const int r = idx >> 6, n = idx & 63;
        const float2 e = g_w64[((r & 63) * n) & 63];
        uint16_t p[PIECES];
        split_pieces<FMT, PIECES>(r < 64 ? e.x : (SIGN > 0 ? e.y : -e.y), p);
        const uint32_t off = kmajor_off(r, n, 64);
#pragma unroll
        for (int q = 0; q < PIECES; ++q) *reinterpret_cast<uint16_t*>(a + q * TCR_A_BYTES + off) = p[q];
    }
}

// D1 = A Bre^T, D2 = A Bim^T, each the sum of the piece products of order <= 1
// (2 pieces: 3 products) or <= 2 (3 pieces: 6 products), 4 K-steps each; then
// commit to mbar
template <int FMT, int PIECES>
__device__ __forceinline__ void issue_split_gemm_k64(uint32_t tmem_d, uint32_t a, uint32_t b, uint32_t mbar) {
    constexpr uint32_t idesc = idesc_f16(FMT, 128, 64);
    constexpr int NT = PIECES == 3 ? 6 : 3;
    constexpr int ta[6] = {0, 0, 1, 0, 2, 1};           // piece of A, of B in each product
    constexpr int tb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        const uint32_t bp = b + part * PIECES * TCR_B_BYTES;
#pragma unroll
        for (int term = 0; term < NT; ++term)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                tc_mma(tmem_d + 64 * part, smem_desc(a + ta[term] * TCR_A_BYTES + ks * 256, 128, 1024),
                       smem_desc(bp + tb[term] * TCR_B_BYTES + ks * 256, 128, 1024), idesc, (term | ks) != 0);
    }
    tc_commit(mbar);
}

// Kinds of 4096-point transform the kernel runs (one per launch):
//   TCM_ROWS_*  steps 2-3: NVMT gather (linear / Keys cubic) of a spectrum row,
//               sign +1, centred in x' and m, in place on the row;
//   TCM_R2C     step 1: two real image columns x, x+1 (zero-expanded rows) as one
//               complex sequence, sign -1, split into their two half spectra; the
//               image comes column-major ([batch][W][H], a transposed copy), so a
//               column pair is two contiguous rows;
//   TCM_C2R     step 4: the Hermitian halves of map columns s, s+1 as one complex
//               spectrum, sign +1, scaled by 1/H', real and imaginary parts to
//               the two map columns, written column-major ([batch][S][H'], to be
//               transposed into the map).
enum { TCM_ROWS_LINEAR = 0, TCM_ROWS_CUBIC = 1, TCM_R2C = 2, TCM_C2R = 3 };

struct TcArgs {
    float2* ws;             // spectrum / G rows [batch][L][S]
    const float* img;       // TCM_R2C input, column-major [batch][W][H]
    float* map;             // TCM_C2R output, column-major [batch][S][H']
    int W, H, Hp, L, S, row0, total;
    unsigned* err;
    long long wait;         // bound of each wait for the GEMMs, SM cycles
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem_src) : "memory");
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(TcPrec<PREC>::THREADS, 1)
k_tc4096(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    using P = TcPrec<PREC>;
    constexpr int FMT = P::FMT, PIECES = P::PIECES, GROUPS = P::GROUPS;
    constexpr int N = TCR_S, T = TCR_GT;
    constexpr int SIGN = MODE == TCM_R2C ? -1 : 1;
    constexpr bool ROWS = MODE == TCM_ROWS_LINEAR || MODE == TCM_ROWS_CUBIC;
    const int g = threadIdx.x / TCR_GT, gt = threadIdx.x % TCR_GT;   // group, thread in group
    const int warp = gt >> 5, lane = gt & 31;          // warp in group = TMEM lane quarter
    unsigned char* aop = sm;                            // DFT matrix pieces
    unsigned char* bop = aop + PIECES * TCR_A_BYTES + g * P::GROUP_BYTES;   // [Re pieces | Im pieces]
    float* stage = reinterpret_cast<float*>(bop + 2 * PIECES * TCR_B_BYTES);   // tcr_sw layout
    float2* zin = reinterpret_cast<float2*>(stage);                      // staged input (aliases stage)
    float2* tw64 = reinterpret_cast<float2*>(aop + PIECES * TCR_A_BYTES + GROUPS * P::GROUP_BYTES);
    float2* tw4k = tw64 + 64;
    __shared__ uint64_t mbar[TCR_MAXG];
    __shared__ uint32_t tmem_base;
    __shared__ float red[TCR_MAXG][4], red2[TCR_MAXG][4];
    __shared__ float2 nyq[TCR_MAXG];                    // TCM_C2R: real parts of the two columns' row H'/2
    const int bar = 1 + g;                              // named barrier of the group

    build_dft_matrix_k64<FMT, PIECES, SIGN>(aop);
    if (threadIdx.x < 64) {
        tw64[threadIdx.x] = g_w64[threadIdx.x];
        tw4k[threadIdx.x] = g_w4096[threadIdx.x];
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < GROUPS; ++j) mbar_init(smem_u32(&mbar[j]), 1);
    if (threadIdx.x < 32) {
        tc_alloc(smem_u32(&tmem_base), 512);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base + 128 * g;         // this group's D1 (+0) and D2 (+64)
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    const uint32_t mb = smem_u32(&mbar[g]);
    uint32_t parity = 0;
    const int r = 32 * warp + lane;                     // accumulator row this thread reads back

    auto group_max = [&](float v) -> float {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[g][warp] = v;
        group_sync(bar);
        const float m = fmaxf(fmaxf(red[g][0], red[g][1]), fmaxf(red[g][2], red[g][3]));
        group_sync(bar);
        return m;
    };
    auto group_sum2 = [&](float2 v) -> float2 {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        if (lane == 0) {
            red[g][warp] = v.x;
            red2[g][warp] = v.y;
        }
        group_sync(bar);
        const float2 t = make_float2((red[g][0] + red[g][1]) + (red[g][2] + red[g][3]),
                                     (red2[g][0] + red2[g][1]) + (red2[g][2] + red2[g][3]));
        group_sync(bar);
        return t;
    };
    // issue the split GEMMs on the group's operands and wait; group-uniform result
    auto gemm = [&]() -> bool {
        fence_async_smem();
        group_sync(bar);
        tc_fence_after();
        if (gt == 0) issue_split_gemm_k64<FMT, PIECES>(tmem, smem_u32(aop), smem_u32(bop), mb);
        bool ok = mbar_wait(mb, parity, a.wait);
        if (!ok) {
            atomicOr(a.err, 1u);
            mbar_wait(mb, parity);                      // let our own MMAs drain (default bound)
        }
        parity ^= 1u;
        tc_fence_after();
        return !group_sync_or(bar, !ok);
    };
    // stage rows 0..63 = Re y, 64..127 = Im y from D1, D2; returns the max |component|
    auto read_d = [&]() -> float {
#pragma unroll 1
        for (int c16 = 0; c16 < 4; ++c16) {
            float d[16];
            tc_ld16(tmem + lane_off + 16 * c16, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[tcr_sw(r, 16 * c16 + j)] = d[j];
        }
        group_sync(bar);
        // thread r < 64: Im y[r] = D2[r] + D1[r + 64]; thread r >= 64: Re y[r - 64] = D1[r - 64] - D2[r]
        const int o = r < 64 ? r + 64 : r - 64;
        const float sg = r < 64 ? 1.f : -1.f;
        float mx = 0.f;
#pragma unroll 1
        for (int c16 = 0; c16 < 4; ++c16) {
            float d[16];
            tc_ld16(tmem + lane_off + 64 + 16 * c16, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = tcr_sw(o, 16 * c16 + j);
                const float v = fmaf(sg, d[j], stage[i]);
                stage[i] = v;
                mx = fmaxf(mx, fabsf(v));
            }
        }
        tc_fence_before();
        return mx;
    };
    // y[k], k = k2 + 64 k1, from the stage after the second GEMM
    auto y_at = [&](int k) -> float2 {
        return make_float2(stage[tcr_sw(k >> 6, k & 63)], stage[tcr_sw((k >> 6) + 64, k & 63)]);
    };

    for (int job = blockIdx.x * GROUPS + g; job < a.total; job += gridDim.x * GROUPS) {
        // ---- stage the input and bound its components
        float mx = 0.f;
        float2 mean = make_float2(0.f, 0.f);            // TCM_R2C: subtracted column means
        int l = 0, img = 0, col = 0;
        if constexpr (ROWS) {
            l = job % a.L;
            float2* row = a.ws + (size_t)job * N;      // row l of image job / L
            if (l == 0) {                               // the DC row is zero
                for (int k = gt; k < N; k += T) row[k] = make_float2(0.f, 0.f);
                continue;
            }
            for (int i = gt; i < a.W / 2; i += T) cp_async16(zin + 2 * i, row + 2 * i);
            cp_async_wait_all();
            for (int i = gt; i < a.W / 2; i += T) {     // this thread's own copies
                const float4 v = *reinterpret_cast<const float4*>(zin + 2 * i);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
        } else if constexpr (MODE == TCM_R2C) {
            img = job / (a.W / 2);
            col = 2 * (job - img * (a.W / 2));
            float* za = reinterpret_cast<float*>(zin);  // column col, zero-expanded to N rows
            float* zb = za + N;                         // column col + 1
            const float* ra = a.img + ((size_t)img * a.W + col) * a.H;
            const float* rb = ra + a.H;
            if (((a.row0 | a.H) & 3) == 0) {            // 16-byte copies
                for (int i = gt; i < N / 4; i += T) {
                    const int y = 4 * i, rr = y - a.row0;
                    if (rr >= 0 && rr < a.H) {
                        cp_async16(za + y, ra + rr);
                        cp_async16(zb + y, rb + rr);
                    } else {
                        *reinterpret_cast<float4*>(za + y) = make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4*>(zb + y) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            } else {
                for (int y = gt; y < N; y += T) {
                    const int rr = y - a.row0;
                    if (rr >= 0 && rr < a.H) {
                        cp_async4(za + y, ra + rr);
                        cp_async4(zb + y, rb + rr);
                    } else {
                        za[y] = 0.f;
                        zb[y] = 0.f;
                    }
                }
            }
            cp_async_wait_all();
            group_sync(bar);
            // the column means (a constant shift changes only Z[0]; it is added back
            // below), so that the split operands carry the columns' variation
            // rather than their mean level
            float sa = 0.f, sb = 0.f;
            for (int y = gt; y < N; y += T) {
                sa += za[y];
                sb += zb[y];
            }
            const float2 tot = group_sum2(make_float2(sa, sb));
            mean = make_float2(tot.x * (1.f / N), tot.y * (1.f / N));
            for (int y = gt; y < N; y += T) mx = fmaxf(mx, fmaxf(fabsf(za[y] - mean.x), fabsf(zb[y] - mean.y)));
        } else {
            img = job / (a.S / 2);
            col = 2 * (job - img * (a.S / 2));
            const float2* src = a.ws + (size_t)img * a.L * a.S + col;
            float4* gst = reinterpret_cast<float4*>(zin);
            for (int ll = gt; ll < N / 2; ll += T) cp_async16(gst + ll, src + (size_t)ll * a.S);
            if (gt == 0) {
                const float2 u = src[(size_t)(N / 2) * a.S], v = src[(size_t)(N / 2) * a.S + 1];
                nyq[g] = make_float2(u.x, v.x);
                mx = fmaxf(fabsf(u.x), fabsf(v.x));
            }
            cp_async_wait_all();
            for (int ll = gt; ll < N / 2; ll += T) {
                const float4 v = gst[ll];
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
        }
        mx = group_max(mx);
        if constexpr (MODE == TCM_ROWS_CUBIC) mx *= 1.25f;          // sum of |Keys weights| <= 1.25
        if constexpr (MODE == TCM_C2R) mx *= 2.f;                    // |A +- i B| components <= 2 max
        const int e1 = mx > 0.f ? ilogbf(mx) : 0;
        const float s1 = ldexpf(1.f, 10 - e1);

        // ---- GEMM 1 operand row n1: x[n1 + 64 n2], n2 = 8 kg .. 8 kg + 7
        if constexpr (ROWS) {
            const int den = 2 * l;
            const float inv = 1.f / (float)den;
            const int step = 64 * a.Hp;                 // n advances by 64 per n2
            const int sA = step / den, sB = step - sA * den;
            const int halfW = a.W >> 1;
            const float2 zero = make_float2(0.f, 0.f);
            for (int item = gt; item < 512; item += T) {
                const int rr = item & 63, kg = item >> 6;       // a warp: 32 operand rows, one K run
                const int n0 = rr + 512 * kg;
                const int num = (n0 - N / 2) * a.Hp;
                int qf = floor_div(num, den), rem = num - qf * den;
                float re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float fr = (float)rem * inv;
                    const int cc = qf + halfW;
                    float2 acc;
                    if constexpr (MODE == TCM_ROWS_LINEAR) {
                        const float2 a0 = (unsigned)cc < (unsigned)a.W ? zin[cc] : zero;
                        const float2 a1 = (unsigned)(cc + 1) < (unsigned)a.W ? zin[cc + 1] : zero;
                        acc = make_float2(fmaf(fr, a1.x - a0.x, a0.x), fmaf(fr, a1.y - a0.y, a0.y));
                    } else {
                        acc = zero;
#pragma unroll
                        for (int d = -1; d <= 2; ++d) {
                            const float2 v = (unsigned)(cc + d) < (unsigned)a.W ? zin[cc + d] : zero;
                            const float w = keys_w(fr - (float)d);
                            acc.x = fmaf(w, v.x, acc.x);
                            acc.y = fmaf(w, v.y, acc.y);
                        }
                    }
                    const float sg = (rr & 1) ? -s1 : s1;         // (-1)^n, n = rr + 64 (8 kg + j)
                    re[j] = acc.x * sg;
                    im[j] = acc.y * sg;
                    rem += sB;
                    qf += sA;
                    if (rem >= den) { rem -= den; qf += 1; }
                }
                put8<FMT, PIECES>(bop, rr, kg, re, im);
            }
        } else {
            const float4* gst = reinterpret_cast<const float4*>(zin);
            for (int item = gt; item < 512; item += T) {
                const int rr = item & 63, kg = item >> 6;       // a warp: 32 operand rows, one K run
                float re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = rr + 64 * (8 * kg + j);
                    float2 z;
                    if constexpr (MODE == TCM_R2C) {
                        const float* za = reinterpret_cast<const float*>(zin);
                        z = make_float2(za[n] - mean.x, za[N + n] - mean.y);
                    } else {
                        const int q = n <= N / 2 ? n : N - n;
                        if (q == N / 2) {
                            z = nyq[g];
                        } else {
                            const float4 v = gst[q];                        // (A, B) of row q
                            if (q == 0) z = make_float2(v.x, v.z);          // Re A + i Re B
                            else z = n <= N / 2 ? make_float2(v.x - v.w, v.y + v.z)     // A + i B
                                                : make_float2(v.x + v.w, v.z - v.y);    // conj A + i conj B
                        }
                    }
                    re[j] = z.x * s1;
                    im[j] = z.y * s1;
                }
                put8<FMT, PIECES>(bop, rr, kg, re, im);
            }
        }
        if (!gemm()) break;
        mx = group_max(read_d());                       // also orders the stage writes before the reads below
        const int e2 = mx > 0.f ? ilogbf(mx) : 0;
        const float s2 = ldexpf(1.f, 10 - e2);
        // ---- twiddle A[k2][n1] (rows k2 / k2 + 64 of stage) and write GEMM 2's operand row k2
        for (int item = gt; item < 512; item += T) {
            const int k2 = item & 63, kg = item >> 6;
            float re[8], im[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n1 = 8 * kg + j;
                const int t = n1 * k2;                  // < 4096
                float2 w = cmul(tw64[t >> 6], tw4k[t & 63]);         // exp(+2 pi i t / 4096)
                if constexpr (SIGN < 0) w.y = -w.y;
                const float x = stage[tcr_sw(k2, n1)], y = stage[tcr_sw(k2 + 64, n1)];
                re[j] = (x * w.x - y * w.y) * s2;
                im[j] = (x * w.y + y * w.x) * s2;
            }
            put8<FMT, PIECES>(bop, k2, kg, re, im);
        }
        if (!gemm()) break;
        read_d();
        group_sync(bar);
        const float un = ldexpf(1.f, e1 + e2 - 20);
        // ---- results
        if constexpr (ROWS) {
            float2* row = a.ws + (size_t)job * N;
            for (int k = gt; k < N; k += T) {
                const float2 y = y_at(k);
                const float sg = ((k + N / 2) & 1) ? -un : un;
                row[k] = make_float2(y.x * sg, y.y * sg);
            }
        } else if constexpr (MODE == TCM_R2C) {
            // half spectra of columns col, col + 1: F_a = (Z[l] + conj Z[N-l]) / 2,
            // F_b = (Z[l] - conj Z[N-l]) / (2 i)
            float2* dst = a.ws + (size_t)img * a.L * a.S + col;
            for (int ll = gt; ll <= N / 2; ll += T) {
                float2 zl = y_at(ll), zm = y_at((N - ll) & (N - 1));
                zl = make_float2(zl.x * un, zl.y * un);
                zm = make_float2(zm.x * un, zm.y * un);
                if (ll == 0) {                          // Z[0] of the unshifted columns
                    zl = make_float2(zl.x + N * mean.x, zl.y + N * mean.y);
                    zm = zl;
                }
                *reinterpret_cast<float4*>(dst + (size_t)ll * a.S) =
                    make_float4(0.5f * (zl.x + zm.x), 0.5f * (zl.y - zm.y), 0.5f * (zl.y + zm.y), -0.5f * (zl.x - zm.x));
            }
        } else {
            float* da = a.map + ((size_t)img * a.S + col) * a.Hp;    // column-major: map column col
            float* db = da + a.Hp;                                    // and col + 1
            const float sc = un / (float)a.Hp;
            for (int t = gt; t < N; t += T) {
                const float2 y = y_at(t);
                da[t] = y.x * sc;
                db[t] = y.y * sc;
            }
        }
        group_sync(bar);                                // stage is the next job's input
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc_dealloc(tmem_base, 512);
}

template <int PREC, int MODE>
static cudaError_t go_tc(const TcArgs& a, cudaStream_t st) {
    using P = TcPrec<PREC>;
    static_assert(P::SMEM + 1024 <= 232448, "shared memory of one block");
    cudaError_t e = cudaFuncSetAttribute(k_tc4096<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int blocks = (a.total + P::GROUPS - 1) / P::GROUPS;
    if (blocks == 0) return cudaSuccess;
    k_tc4096<PREC, MODE><<<blocks < sms ? blocks : sms, P::THREADS, P::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t go_tc_prec(int prec, const TcArgs& a, cudaStream_t st) {
    switch (prec) {
        case FT_PRECISION_BF16X3: return go_tc<FT_PRECISION_BF16X3, MODE>(a, st);
        case FT_PRECISION_FP16X3: return go_tc<FT_PRECISION_FP16X3, MODE>(a, st);
        case FT_PRECISION_BF16X6: return go_tc<FT_PRECISION_BF16X6, MODE>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_nvmt_rows_tc4096(float2* ws, int W, int Hp, int L, int interp, int prec, unsigned* err,
                                    long long wait, int batch, cudaStream_t st) {
    if (W <= 0 || W > TCR_S || (W & 1) || wait < 0) return cudaErrorInvalidValue;
    cudaError_t e = ensure_w64();
    if (e != cudaSuccess) return e;
    TcArgs a{ws, nullptr, nullptr, W, 0, Hp, L, TCR_S, 0, batch * L, err, wait};
    return interp == FT_INTERP_LINEAR ? go_tc_prec<TCM_ROWS_LINEAR>(prec, a, st)
                                      : go_tc_prec<TCM_ROWS_CUBIC>(prec, a, st);
}

cudaError_t launch_col_r2c_tc4096(const float* img_cm, int H, int W, int row0, float2* ws, int L, int S, int prec,
                                  unsigned* err, long long wait, int batch, cudaStream_t st) {
    if (H <= 0 || H > TCR_S || W <= 0 || (W & 1) || L != TCR_S / 2 + 1 || S < W || wait < 0)
        return cudaErrorInvalidValue;
    cudaError_t e = ensure_w64();
    if (e != cudaSuccess) return e;
    TcArgs a{ws, img_cm, nullptr, W, H, TCR_S, L, S, row0, batch * (W / 2), err, wait};
    return go_tc_prec<TCM_R2C>(prec, a, st);
}

cudaError_t launch_col_c2r_tc4096(const float2* ws, int L, int S, float* map_cm, int prec, unsigned* err,
                                  long long wait, int batch, cudaStream_t st) {
    if (L != TCR_S / 2 + 1 || S <= 0 || (S & 1) || wait < 0) return cudaErrorInvalidValue;
    cudaError_t e = ensure_w64();
    if (e != cudaSuccess) return e;
    TcArgs a{const_cast<float2*>(ws), nullptr, map_cm, 0, 0, TCR_S, L, S, 0, batch * (S / 2), err, wait};
    return go_tc_prec<TCM_C2R>(prec, a, st);
}
