// Register-resident Stockham FFT with compile-time schedules.
//
// For the lengths below every thread of a transform holds E elements (16, or 12
// when N has a factor 3) in registers; a transform of length N uses T = N / E
// threads, and a block runs B transforms side by side (transform f's sample n
// lives at smem[spos(n) * B + f]).  A pass with radix R and P = product of the
// earlier radices does, for butterfly i in [0, N/R) with k = i mod P:
//     inputs x[i + q N/R] * w^{q k N/(P R)},  q < R   (w = exp(SIGN 2 pi i / N))
//     radix-R DFT in registers
//     outputs y[(i - k) R + k + q P]
// so the result comes out in natural order (self-sorting).  Each pass costs one
// shared-memory round trip; the first pass loads and the last pass stores
// through caller code, which lets the column and row kernels read and write
// global memory directly.  All index arithmetic is by compile-time constants.
//
// Twiddles come from a per-length table (FP64 values rounded to FP32, built on
// the host): for pass s >= 1, row k of a full table holds w_k^q at column q
// (q = 0 .. R-1), w_k = exp(-2 pi i k / (P R)); row k of a seed table holds
// only w_k^e for the exponents e = 1, 2, 4, 8 below R (1, 2 for R = 3), and a
// thread builds the other powers as products of at most four seeds (a few
// FP32 roundings).  Rows are padded to an even length so that pairs load as
// float4.  A radix-16 group reads 8 float4 of a full row against 2 of a seed
// row and 11 complex products: the row kernels (steps 2-3, scattered rows k
// per lane) run faster on seed tables (103 against 112 us per 64 x 1024^2),
// the column kernels on full ones (step 4: 121 against 128 us).
#pragma once

#include "ft_internal.cuh"

__host__ __device__ constexpr bool fs_has(int N) {
    return N == 128 || N == 256 || N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192 ||
           N == 192 || N == 384 || N == 768 || N == 1536;
}
__host__ __device__ constexpr int fs_E(int N) { return N % 3 == 0 ? 12 : 16; }
__host__ __device__ constexpr int fs_T(int N) { return N / fs_E(N); }
__host__ __device__ constexpr int fs_nst(int N) {
    return N == 128 ? 2 : N == 256 ? 2 : N == 512 ? 3 : N == 1024 ? 3 : N == 2048 ? 3 : N == 4096 ? 3
         : N == 8192 ? 4 : N == 192 ? 4 : N == 384 ? 5 : N == 768 ? 5 : N == 1536 ? 6 : 0;
}
__host__ __device__ constexpr int fs_radix(int N, int s) {
    return N == 128 ? (s == 0 ? 16 : 8)
         : N == 256 ? 16
         : N == 512 ? (s == 0 ? 16 : s == 1 ? 8 : 4)
         : N == 1024 ? (s < 2 ? 16 : 4)
         : N == 2048 ? (s < 2 ? 16 : 8)
         : N == 4096 ? 16
         : N == 8192 ? (s < 3 ? 16 : 2)
         : N == 192 ? (s < 3 ? 4 : 3)
         : N == 384 ? (s < 3 ? 4 : s == 3 ? 2 : 3)
         : N == 768 ? (s < 4 ? 4 : 3)
         : N == 1536 ? (s < 4 ? 4 : s == 4 ? 2 : 3)
         : 0;
}
__host__ __device__ constexpr int fs_P(int N, int s) {
    int p = 1;
    for (int j = 0; j < s; ++j) p *= fs_radix(N, j);
    return p;
}
// seed powers of a pass with radix R (exponents 1 << j, j < fs_nseed(R)) and the
// twiddle row stride of a full or a seed table, rounded up to even (16-byte rows)
__host__ __device__ constexpr int fs_nseed(int R) { return R == 16 ? 4 : R == 8 ? 3 : R == 2 ? 1 : 2; }
__host__ __device__ constexpr int fs_rs(int R, bool seed) { return ((seed ? fs_nseed(R) : R) + 1) & ~1; }
__host__ __device__ constexpr int fs_twoff(int N, int s, bool seed) {
    int o = 0;
    for (int j = 1; j < s; ++j) o += fs_P(N, j) * fs_rs(fs_radix(N, j), seed);
    return o;
}
__host__ __device__ constexpr int fs_twsize(int N, bool seed) { return fs_twoff(N, fs_nst(N), seed); }
// transforms per block for the column R2C kernels (512 threads; for N >= 4096,
// 1024 threads so that a block still reads 4 column pairs = 32-byte row
// segments), the column C2R kernel (256 threads, at least 4 column pairs, so
// 512 threads for N = 1536, 2048; for N = 1024 512 threads, 8 column pairs:
// with the tile maxima of ft_detect 121 us per 64 x 1024^2 against 124 us with
// 256, and the peak pass is faster on the 16 x 16 tiles that gives) and the row
// kernels (128 threads: at N = 1024, 2 rows per block run 116 us per
// 64 x 1024^2, 4 rows 128 us, 1 row 142 us)
__host__ __device__ constexpr int fs_clampB(int v, int hi) { return v < 1 ? 1 : (v > hi ? hi : v); }
__host__ __device__ constexpr int fs_Bcol(int N) { return fs_T(N) >= 256 ? 1024 / fs_T(N) : fs_clampB(512 / fs_T(N), 32); }
__host__ __device__ constexpr int fs_Bc2r(int N) {
    return fs_T(N) >= 256 ? 1024 / fs_T(N)
                          : fs_clampB(N == 1024 ? 512 / fs_T(N) : (256 / fs_T(N) < 4 ? 4 : 256 / fs_T(N)), 32);
}
__host__ __device__ constexpr int fs_Brow(int N) { return fs_clampB(128 / fs_T(N), 16); }
// padded shared-memory slot of sample n (one spare slot every 16 samples
// spreads the strided stores of the first pass over the banks)
__host__ __device__ constexpr int spos(int n) { return n + (n >> 4); }
__host__ __device__ constexpr int fs_slots(int N) { return spos(N - 1) + 1; }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int SIGN>
__device__ __forceinline__ float2 tw_sign(float2 w) { return SIGN > 0 ? make_float2(w.x, -w.y) : w; }

// w[q] = w_k^q (conjugated for SIGN > 0), q = 1 .. R-1, from the seed row at wp
template <int R, int SIGN>
__device__ __forceinline__ void tw_powers(const float4* __restrict__ wp, float2 (&w)[R]) {
    const float4 a = __ldg(wp);
    w[1] = tw_sign<SIGN>(make_float2(a.x, a.y));
    if constexpr (R == 3) {
        w[2] = tw_sign<SIGN>(make_float2(a.z, a.w));
    } else if constexpr (R >= 4) {
        w[2] = tw_sign<SIGN>(make_float2(a.z, a.w));
        w[3] = cmul(w[1], w[2]);
        if constexpr (R >= 8) {
            const float4 b = __ldg(wp + 1);
            w[4] = tw_sign<SIGN>(make_float2(b.x, b.y));
            w[5] = cmul(w[1], w[4]);
            w[6] = cmul(w[2], w[4]);
            w[7] = cmul(w[3], w[4]);
            if constexpr (R == 16) {
                w[8] = tw_sign<SIGN>(make_float2(b.z, b.w));
#pragma unroll
                for (int q = 9; q < 16; ++q) w[q] = cmul(w[q - 8], w[8]);
            }
        }
    }
    static_assert(R == 2 || R == 3 || R == 4 || R == 8 || R == 16, "radix without seed powers");
}

// radix-16 as 4 x 4 with the internal twiddles exp(SIGN 2 pi i m / 16)
template <int SIGN>
struct Dft<16, SIGN> {
    __device__ __forceinline__ static void run(float2* u) {
        const float c1 = 0.92387953251128675613f;   // cos(pi/8)
        const float s1 = 0.38268343236508977173f;   // sin(pi/8)
        const float r = 0.70710678118654752440f;    // sqrt(2)/2
        float2 a[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 t[4] = {u[n2], u[4 + n2], u[8 + n2], u[12 + n2]};
            Dft<4, SIGN>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
        }
        const float2 w1 = make_float2(c1, SIGN * s1), w2 = make_float2(r, SIGN * r);
        const float2 w3 = make_float2(s1, SIGN * c1), w6 = make_float2(-r, SIGN * r);
        const float2 w9 = make_float2(-c1, -SIGN * s1);
        a[1][1] = cmul(a[1][1], w1);
        a[1][2] = cmul(a[1][2], w2);
        a[1][3] = cmul(a[1][3], w3);
        a[2][1] = cmul(a[2][1], w2);
        a[2][2] = cmul_si<SIGN>(a[2][2]);
        a[2][3] = cmul(a[2][3], w6);
        a[3][1] = cmul(a[3][1], w3);
        a[3][2] = cmul(a[3][2], w6);
        a[3][3] = cmul(a[3][3], w9);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            Dft<4, SIGN>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) u[k1 + 4 * k2] = t[k2];
        }
    }
};

// SEED: the twiddle table is a seed table (the row kernels' tables), else full
template <int N, int SIGN, int B, bool SEED = false>
struct FastFft {
    static constexpr int E = fs_E(N);
    static constexpr int T = N / E;
    static constexpr int NS = fs_nst(N);
    static constexpr int SLOTS = fs_slots(N) * B;      // float2 slots of shared memory

    // sample index of element (m, q) of pass s for thread t of a transform
    template <int s>
    __device__ __forceinline__ static int in_pos(int t, int m, int q) {
        return t + m * T + q * (N / fs_radix(N, s));
    }
    // sample index of output element (m, q) of the last pass
    __device__ __forceinline__ static int out_pos(int t, int m, int q) {
        return t + m * T + q * (N / fs_radix(N, NS - 1));
    }

    template <int s>
    __device__ __forceinline__ static void compute(float2 (&v)[E], int t, const float2* __restrict__ stw) {
        constexpr int R = fs_radix(N, s), P = fs_P(N, s), G = E / R;
#pragma unroll
        for (int m = 0; m < G; ++m) {
            if constexpr (P > 1 && SEED) {
                constexpr int RS = fs_rs(R, true);
                const int k = (t + m * T) % P;
                float2 w[R];
                tw_powers<R, SIGN>(reinterpret_cast<const float4*>(stw + fs_twoff(N, s, true) + k * RS), w);
#pragma unroll
                for (int q = 1; q < R; ++q) v[m * R + q] = cmul(v[m * R + q], w[q]);
            } else if constexpr (P > 1) {
                constexpr int RS = fs_rs(R, false);
                const int k = (t + m * T) % P;
                const float4* w = reinterpret_cast<const float4*>(stw + fs_twoff(N, s, false) + k * RS);
#pragma unroll
                for (int h = 0; h < RS / 2; ++h) {
                    const float4 ww = __ldg(w + h);
                    if (2 * h >= 1 && 2 * h < R)
                        v[m * R + 2 * h] = cmul(v[m * R + 2 * h], tw_sign<SIGN>(make_float2(ww.x, ww.y)));
                    if (2 * h + 1 < R)
                        v[m * R + 2 * h + 1] = cmul(v[m * R + 2 * h + 1], tw_sign<SIGN>(make_float2(ww.z, ww.w)));
                }
            }
            Dft<R, SIGN>::run(&v[m * R]);
        }
    }

    template <int s>
    __device__ __forceinline__ static void store(const float2 (&v)[E], float2* sm, int t, int f) {
        constexpr int R = fs_radix(N, s), P = fs_P(N, s), G = E / R;
#pragma unroll
        for (int m = 0; m < G; ++m) {
            const int i = t + m * T;
            const int k = i % P;
            const int j = (i - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (FT_IN(spos(j + q * P) * B + f, SLOTS, FT_DBG_FFT_SLOT)) sm[spos(j + q * P) * B + f] = v[m * R + q];
        }
    }

    template <int s>
    __device__ __forceinline__ static void load(float2 (&v)[E], const float2* sm, int t, int f) {
        constexpr int R = fs_radix(N, s), G = E / R;
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int k = spos(in_pos<s>(t, m, q)) * B + f;
                v[m * R + q] = FT_IN(k, SLOTS, FT_DBG_FFT_SLOT) ? sm[k] : make_float2(0.f, 0.f);
            }
    }

    // The barriers of run<s> for the threads of a block that hold no transform of
    // this length (a block whose stages use transforms of different lengths).
    template <int s>
    __device__ __forceinline__ static void idle() {
        if constexpr (s + 1 < NS) {
            __syncthreads();
            __syncthreads();
            idle<s + 1>();
        }
    }

    // Passes s .. NS-1.  On entry v holds the inputs of pass s in (m, q) order;
    // on return it holds the outputs of the last pass, element (m, q) being the
    // sample out_pos(t, m, q).  Every thread of the block must call it; it leaves
    // shared memory free to reuse (the last barrier follows the last read).
    template <int s>
    __device__ __forceinline__ static void run(float2 (&v)[E], float2* sm, int t, int f,
                                               const float2* __restrict__ stw) {
        compute<s>(v, t, stw);
        if constexpr (s + 1 < NS) {
            store<s>(v, sm, t, f);
            __syncthreads();
            load<s + 1>(v, sm, t, f);
            __syncthreads();
            run<s + 1>(v, sm, t, f, stw);
        }
    }
};

// launchers of the fixed-length kernels (k_fast.cu); they return
// cudaErrorNotSupported when N has no schedule

// (pdl: launched with programmatic stream serialisation, the blocks waiting for
// the predecessor before they read or write; follows_peak (with pdl): the
// predecessor is the peak pass of the previous batch of ft_detect_batches, not
// waited for (see k_col_r2c_fast); err, wait: with err given, the image columns
// are staged through tensor copies whose bounded waits set bit 3 of *err when
// they run out)
cudaError_t launch_col_r2c_fast(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img,
                                int row0, const FftLen& f, float2* out, int out_pitch, size_t out_img,
                                float end_scale, float mid_scale, int batch, cudaStream_t st, bool pdl = false,
                                bool follows_peak = false, unsigned* err = nullptr,
                                long long wait = FT_WAIT_CYCLES);
// the adjoint of step 4 with the input gradient computed from the map and the
// target of the gradient workload (k_col_r2c_loss_fast); partial gets
// col_r2c_loss_blocks() floats per image
int col_r2c_loss_blocks(const FftLen& f, int ncols);
// (err, wait: with err given, the map columns are staged through tensor copies
// whose bounded waits set bit 3 of *err when they run out)
cudaError_t launch_col_r2c_loss_fast(const float* map, const float* target, int ncols, const FftLen& f,
                                     float2* out, int out_pitch, size_t out_img, float end_scale, float mid_scale,
                                     float scale, float gscale, float* partial, int batch, cudaStream_t st,
                                     unsigned* err = nullptr, long long wait = FT_WAIT_CYCLES);
// tmax (may be NULL; only with row0 = 0 and rows_out = N): the maxima of |out| per
// tile of c2r_tile_shape rows x columns, [batch][N / rows][ceil(ncols / cols)] as
// float bits
// (err, wait: with err given, the staging goes through tensor copies whose
// bounded waits set bit 2 of *err when they run out; without, cp.async)
cudaError_t launch_col_c2r_fast(const float2* in, int ncols, int in_pitch, size_t in_img,
                                const FftLen& f, float mid_scale, float* out, int row0, int rows_out,
                                int out_pitch, size_t out_img, float out_scale, int batch,
                                cudaStream_t st, unsigned* tmax = nullptr, bool pdl = false,
                                unsigned* err = nullptr, long long wait = FT_WAIT_CYCLES);
// tiles of the tile maxima of launch_col_c2r_fast for length N: rows x cols
// cells, bands = N / rows tiles per column block; false without a schedule.
// A tile is 256 cells: 128 / B rows of one column block of 2B columns.
__host__ __device__ constexpr int c2r_tile_rows(int N) { return 128 / fs_Bc2r(N); }
bool c2r_tile_shape(int N, int* rows, int* cols, int* bands);
// (err: bit 1 set when a bulk-copy wait ran out after `wait` SM cycles)
cudaError_t launch_nvmt_rows_fast(float2* ws, int W, int Hp, int L, int interp, const FftLen& fx,
                                  int batch, cudaStream_t st, bool pdl, unsigned* err, long long wait);
cudaError_t launch_nvmt_rows_adjoint_fast(float2* ws, int W, int Hp, int L, int interp,
                                          const FftLen& fx, int batch, cudaStream_t st);
