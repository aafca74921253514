// One block's work of the fixed-length column and row kernels (see k_cols.cu and
// k_rows.cu for what each step computes), built on the register-resident FFT of
// fft_fast.cuh.  The per-plan kernels of k_fast.cu run one of these per CUDA
// block over a uniform batch; the mixed-size batch kernels of k_batch.cu run
// them from a work queue over images of different lengths.  B, the transforms
// per block, is a template parameter: the block has fs_T(N) * B threads.
//  * the column R2C reads its first pass directly from global memory; the
//    other two stage their inputs into shared memory with 16-byte cp.async
//    copies, all in flight at once (C2R: the Hermitian half, each row read once
//    for both n and N - n; rows: the B spectrum rows feeding the NVMT gather);
//    the last pass writes global memory directly where the output order allows;
//  * the NVMT sample x' H' / (2 l) of successive elements of a thread is stepped
//    exactly by adding the precomputed quotient and remainder of
//    (N / R0) H' / (2 l), so the inner loop has no integer division;
//  * the interpolation fraction is remainder * (1 / (2 l)) in FP32 (within one
//    rounding of the exact fraction).
#pragma once

#include "async_copy.cuh"
#include "fft_fast.cuh"

// The last pass of the column R2C and the split of each complex transform (two
// real columns a + i b) into the two half spectra:
//     A[l] = (Z[l] + conj Z[N-l]) / 2,  B[l] = (Z[l] - conj Z[N-l]) / (2 i),
// scaled by end_scale (l = 0, N/2) or mid_scale, written as one float4 per row.
template <int N, int B>
__device__ __forceinline__ void r2c_finish(float2 (&v)[fs_E(N)], float2* sm, int t, int f, const float2* stw,
                                           bool colok, float2* dst, int out_pitch, float end_scale,
                                           float mid_scale) {
    constexpr int E = fs_E(N), T = N / E;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    using F = FastFft<N, -1, B>;
    F::template run<0>(v, sm, t, f, stw);
    // Sample t + T j is the thread's element (j mod GL, j / GL).  Thread t != 0
    // writes l = t + T j (j < E/2) and needs Z[N - l] = Z[(T - t) + T (E - 1 - j)],
    // element E - 1 - j >= E/2 of thread T - t; thread 0 writes l = T j
    // (j <= E/2) and needs Z[N - l], its own element E - j (element 0 for l = 0).
    // So only elements j >= E/2 go through shared memory.
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q)
            if (m + GL * q >= E / 2 && FT_IN(spos(F::out_pos(t, m, q)) * B + f, F::SLOTS, FT_DBG_FFT_SLOT))
                sm[spos(F::out_pos(t, m, q)) * B + f] = v[m * RL + q];
    __syncthreads();
    if (!colok) return;
    auto el = [&](int j) -> float2 { return v[(j % GL) * RL + j / GL]; };
    auto split_z = [&](int l, float2 zl, float2 zm, float s) {
        float4 o;
        o.x = 0.5f * s * (zl.x + zm.x);
        o.y = 0.5f * s * (zl.y - zm.y);
        o.z = 0.5f * s * (zl.y + zm.y);
        o.w = -0.5f * s * (zl.x - zm.x);
        if (FT_IN(l, N / 2 + 1, FT_DBG_R2C_STORE)) *reinterpret_cast<float4*>(dst + (size_t)l * out_pitch) = o;
    };
    // only t = 0 meets the end bins 0 and N/2 (N/2 is a multiple of T)
    if (t != 0) {
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
            const int k = spos(N - t - T * j) * B + f;
            split_z(t + T * j, el(j), FT_IN(k, F::SLOTS, FT_DBG_FFT_SLOT) ? sm[k] : make_float2(0.f, 0.f), mid_scale);
        }
    } else {
        split_z(0, el(0), el(0), end_scale);
#pragma unroll
        for (int j = 1; j < E / 2; ++j) split_z(T * j, el(j), el(E - j), mid_scale);
        split_z(N / 2, el(E / 2), el(E / 2), end_scale);
    }
}

// Step 1 (and the transpose of step 4) for column block bx of one image: real
// columns bx 2B + 2f, + 1 of `in` (rows_in rows, pitch in_pitch floats, first
// row at expanded row row0, zeros elsewhere) -> half spectra out[l][c] (pitch
// out_pitch complex).  The first pass reads global memory directly (8-byte
// loads of the thread's column pair): staging the image tile through shared
// memory first measured slower on GB300 (67 vs 60 us for 32 images of 1024^2).
// TMA: the block's 2B image columns of all N expanded rows arrive by tma_nb
// tensor copies of tma_h rows (tmap: the launch's images as [images][rows_in]
// [ncols] floats, image `img`; rows outside the image and columns past it read
// zeros), waited for on an mbarrier with the bound `wait`; when it runs out, bit
// 3 of *err is set, the block waits (default bound) for its copies and returns
// false without writing; pf_img >= 0: the same boxes of column block pf_bx of
// image pf_img (a block half a resident wave later) are prefetched into L2.
// Otherwise the first pass reads global memory directly.
template <int N, int B, bool TMA = false>
__device__ __forceinline__ bool r2c_block(const float* __restrict__ in, int rows_in, int ncols, int in_pitch,
                                          int row0, const float2* __restrict__ stw, float2* __restrict__ out,
                                          int out_pitch, float end_scale, float mid_scale, int bx, float2* sm,
                                          const CUtensorMap* tmap = nullptr, int tma_h = 0, int tma_nb = 0,
                                          int img = 0, unsigned* err = nullptr, long long wait = FT_WAIT_CYCLES,
                                          int pf_bx = 0, int pf_img = -1) {
    constexpr int E = fs_E(N);
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    using F = FastFft<N, -1, B>;
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = bx * 2 * B + 2 * f;
    const bool colok = c < ncols;
    const float* src = in + c;

    float2 v[E];
    if constexpr (TMA) {
        float* stg = reinterpret_cast<float*>(sm);     // [tma_nb tma_h][2B] floats
        __shared__ uint64_t mbar;
        const uint32_t mb = smem_u32(&mbar);
        if (threadIdx.x == 0) {
            mbar_init(mb, 1);
            mbar_arrive_expect_tx(mb, (uint32_t)(tma_nb * tma_h * 2 * B * sizeof(float)));
            for (int k = 0; k < tma_nb; ++k)
                tma_load_3d(stg + k * tma_h * 2 * B, tmap, bx * 2 * B, k * tma_h - row0, img, mb);
            if (pf_img >= 0)
                for (int k = 0; k < tma_nb; ++k) tma_prefetch_3d(tmap, pf_bx * 2 * B, k * tma_h - row0, pf_img);
        }
        __syncthreads();                               // the mbarrier is initialised
        const bool ok = mbar_wait(mb, 0, wait);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && err) atomicOr(err, 8u);
            mbar_wait(mb, 0);                          // the copies in flight land first
            return false;
        }
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q)
                v[m * R0 + q] = *reinterpret_cast<const float2*>(stg + F::template in_pos<0>(t, m, q) * 2 * B + 2 * f);
        __syncthreads();                               // the staged tile is dead before the first exchange
    } else if (colok && row0 == 0 && rows_in == N) {   // every row is an image row
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const int row = F::template in_pos<0>(t, m, q);
                v[m * R0 + q] = FT_IN(row, rows_in, FT_DBG_R2C_LOAD) && FT_IN(c + 1, ncols, FT_DBG_R2C_LOAD)
                                    ? __ldg(reinterpret_cast<const float2*>(src + (size_t)row * in_pitch))
                                    : make_float2(0.f, 0.f);
            }
    } else {
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const int row = F::template in_pos<0>(t, m, q) - row0;
                float2 x = make_float2(0.f, 0.f);
                if (colok && row >= 0 && row < rows_in && FT_IN(c + 1, ncols, FT_DBG_R2C_LOAD))
                    x = __ldg(reinterpret_cast<const float2*>(src + (size_t)row * in_pitch));
                v[m * R0 + q] = x;
            }
    }
    r2c_finish<N, B>(v, sm, t, f, stw, colok, out + c, out_pitch, end_scale, mid_scale);
    return true;
}

// The part of step 4 after staging, for column block bx of one image: sm holds
// the Hermitian half [N/2 + 1][2B] complex (and serves as the FFT's exchange
// buffer afterwards); arguments as for c2r_block.
template <int N, int B>
__device__ __forceinline__ void c2r_from_stage(float2* sm, int ncols, const float2* __restrict__ stw,
                                               float mid_scale, float* __restrict__ out, int row0, int rows_out,
                                               int out_pitch, float out_scale, unsigned* __restrict__ tmax, int nbx,
                                               int bx) {
    constexpr int E = fs_E(N);
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    using F = FastFft<N, +1, B>;
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = bx * 2 * B + 2 * f;
    const bool colok = c < ncols;
    const float2* stg = sm;
    // sample n = t + T (m + G0 q) comes from row n when m + G0 q < E/2 and from
    // row N - n otherwise (the two agree at n = N/2); the end bins 0 and N/2,
    // which only thread t = 0 holds, enter through their real parts
    float2 v[E];
#pragma unroll
    for (int m = 0; m < G0; ++m)
#pragma unroll
        for (int q = 0; q < R0; ++q) {
            const int n = F::template in_pos<0>(t, m, q);
            const bool up = m + G0 * q < E / 2;
            const int row = up ? n : N - n;
            float4 g = FT_IN(row, N / 2 + 1, FT_DBG_C2R_STAGE)
                           ? *reinterpret_cast<const float4*>(stg + row * 2 * B + 2 * f)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            g.x *= mid_scale; g.y *= mid_scale; g.z *= mid_scale; g.w *= mid_scale;
            v[m * R0 + q] = up ? make_float2(g.x - g.w, g.y + g.z)      // A + i B
                               : make_float2(g.x + g.w, g.z - g.y);     // conj A + i conj B
        }
    if (t == 0) {
        constexpr int mh = (E / 2) % G0, qh = (E / 2) / G0;          // the element of n = N/2
        const float4 g0 = *reinterpret_cast<const float4*>(stg + 2 * f);
        const float4 gh = *reinterpret_cast<const float4*>(stg + (N / 2) * 2 * B + 2 * f);
        v[0] = make_float2(g0.x, g0.z);                               // Re A + i Re B
        v[mh * R0 + qh] = make_float2(gh.x, gh.z);
    }
    __syncthreads();
    F::template run<0>(v, sm, t, f, stw);
    if (tmax) {
        // Tile maxima of |map| for the peak pass: thread t holds rows t + T j,
        // j = m + GL q, of its column pair.  A tile is RS = 128 / B consecutive
        // rows of one band (rows T j + RS u .. T j + RS u + RS - 1, u < T / RS) of
        // the block's 2B columns: 256 cells held, one each, by the 128
        // consecutive threads RS B u .. RS B u + 127, i.e. by whole warps
        // 4u .. 4u + 3.  Every warp reduces its 32 values of band j with one
        // redux.sync (max(|re|, |im|) of the stored, scaled values; NaN counts
        // as 0, like a cell that is never a peak), lane 0 keeps the partial in
        // the exchange buffer, which the FFT no longer reads, and one thread per
        // tile combines its four warps' partials.
        constexpr int NT = fs_T(N) * B;                // threads of the block
        constexpr int NW = NT / 32;
        constexpr int RS = 128 / B, TPB = fs_T(N) / RS;   // tile rows, tiles per band
        static_assert(RS * B == 128 && TPB * RS == fs_T(N), "a tile is 128 threads' values");
        static_assert(E * NW <= FastFft<N, +1, B>::SLOTS * 2, "partial maxima fit the exchange buffer");
        unsigned* part = reinterpret_cast<unsigned*>(sm);  // [E][NW]
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int m = 0; m < GL; ++m)
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const float a = fabsf(v[m * RL + q].x * out_scale), b = fabsf(v[m * RL + q].y * out_scale);
                const unsigned x = __reduce_max_sync(0xffffffffu, colok ? __float_as_uint(fmaxf(fmaxf(a, b), 0.f)) : 0u);
                if (lane == 0) part[(m + GL * q) * NW + warp] = x;
            }
        __syncthreads();
        for (int w = threadIdx.x; w < E * TPB; w += NT) {
            const unsigned* p = part + (w / TPB) * NW + 4 * (w % TPB);
            const unsigned x = max(max(p[0], p[1]), max(p[2], p[3]));
            if (FT_IN(bx, nbx, FT_DBG_C2R_STORE)) tmax[(size_t)w * nbx + bx] = x;
        }
    }
    if (!colok) return;
    // row n of the result goes to output row n - row0 when that is in range
    float* dst = out + c;
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int rr = F::out_pos(t, m, q) - row0;
            if ((unsigned)rr < (unsigned)rows_out && FT_IN(c + 1, ncols, FT_DBG_C2R_STORE))
                *reinterpret_cast<float2*>(dst + (size_t)rr * out_pitch) =
                    make_float2(v[m * RL + q].x * out_scale, v[m * RL + q].y * out_scale);
        }
}

// Step 4 (and the transpose of step 1) for column block bx of one image: the
// Hermitian halves in[l][c] (pitch in_pitch complex, l = 0 .. N/2) of columns
// bx 2B + 2f, + 1 -> rows row0 .. row0 + rows_out - 1 of the length-N real
// results, times out_scale, at out[t - row0][c] (pitch out_pitch floats).
// tmax (may be NULL; only with row0 = 0 and rows_out = N): the maximum of |out|
// of every tile of 128 / B rows x 2B columns, at tmax[tile row * nbx + bx]
// (nbx = column blocks of the image) as float bits.
// TMA: the Hermitian half arrives by nb tensor copies of h rows x 2B complex
// (tmap: the launch's half spectra as [images][rows][in_pitch] 8-byte elements,
// image `img`; rows past N/2 and columns past the tensor read zeros), waited for
// on an mbarrier with the bound `wait` in SM cycles; when a wait runs out, bit 2
// of *err is set, the block waits (default bound) for its copies in flight and
// returns false without writing; pf_img >= 0: the same boxes of column block
// pf_bx of image pf_img (a block half a resident wave later) are prefetched into
// L2.  Otherwise every thread copies 16-byte pieces.
template <int N, int B, bool TMA = false>
__device__ __forceinline__ bool c2r_block(const float2* __restrict__ in, int ncols, int in_pitch,
                                          const float2* __restrict__ stw, float mid_scale, float* __restrict__ out,
                                          int row0, int rows_out, int out_pitch, float out_scale,
                                          unsigned* __restrict__ tmax, int nbx, int bx, float2* sm,
                                          const CUtensorMap* tmap = nullptr, int tma_h = 0, int tma_nb = 0,
                                          int img = 0, unsigned* err = nullptr, long long wait = FT_WAIT_CYCLES,
                                          int pf_bx = 0, int pf_img = -1) {
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = bx * 2 * B + 2 * f;
    const bool colok = c < ncols;

    // stage the Hermitian half (rows 0 .. N/2, 2B complex each) with 16-byte async
    // copies; every row is read once and serves both n and N - n.  Thread (t, f)
    // copies the column pair f of rows t, t + T, ...
    float2* stg = sm;                                  // [N/2 + 1][2B]
    if constexpr (TMA) {
        __shared__ uint64_t mbar;
        const uint32_t mb = smem_u32(&mbar);
        if (threadIdx.x == 0) {
            mbar_init(mb, 1);
            mbar_arrive_expect_tx(mb, (uint32_t)(tma_nb * tma_h * 2 * B * sizeof(float2)));
            for (int k = 0; k < tma_nb; ++k) tma_load_3d(stg + k * tma_h * 2 * B, tmap, bx * 2 * B, k * tma_h, img, mb);
            if (pf_img >= 0)
                for (int k = 0; k < tma_nb; ++k) tma_prefetch_3d(tmap, pf_bx * 2 * B, k * tma_h, pf_img);
        }
        __syncthreads();                               // the mbarrier is initialised
        const bool ok = mbar_wait(mb, 0, wait);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && err) atomicOr(err, 4u);
            mbar_wait(mb, 0);                          // the copies in flight land first
            return false;
        }
    } else {
        const float2* src = in + c + (size_t)t * in_pitch;
        float2* dst = stg + t * 2 * B + 2 * f;
        for (int r = t; r <= N / 2; r += fs_T(N), src += (size_t)fs_T(N) * in_pitch, dst += fs_T(N) * 2 * B) {
            if (colok)
                cp_async16(dst, src);
            else
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    c2r_from_stage<N, B>(sm, ncols, stw, mid_scale, out, row0, rows_out, out_pitch, out_scale, tmax, nbx, bx);
    return true;
}

// row pitch (complex) of the staged spectrum rows: W samples between two zero
// samples on each side (so a clamped tap index needs no bounds test); W + 4
// keeps 16-byte alignment for cp.async and shifts successive rows by 8 banks
__host__ __device__ constexpr int srow_pitch(int W) { return W + 4; }

// Steps 2-3 in place for rows bx B .. bx B + B - 1 of one image's half spectrum
// base[L][N] (W columns of image data per row before, N = n_slope values of G
// after): the NVMT gather with the exact positions x' H' / (2 l), then the
// exp(+j) transform along x'.  Row 0 becomes zero.  Shared memory: the larger
// of the FFT's exchange buffer and B staged rows of srow_pitch(W) complex.
// BULK: each staged row arrives by one bulk copy (the copy engine, not the
// threads' load/store path) completing on an mbarrier, waited for with the
// bound `wait` in SM cycles; when a wait runs out, bit 1 of *err is set, the
// block waits (default bound) for its copies in flight and returns false
// without writing.  Otherwise every thread copies 16-byte pieces (cp.async).
template <int N, int INTERP, int B, bool BULK = false>
__device__ __forceinline__ bool rows_block(float2* __restrict__ base, int W, int Hp, int L,
                                           const float2* __restrict__ stw, int bx, float2* sm,
                                           unsigned* err = nullptr, long long wait = FT_WAIT_CYCLES) {
    constexpr int E = fs_E(N), T = N / E;
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    constexpr int STEPX = N / R0;                      // x' distance between a thread's elements
    using F = FastFft<N, +1, B, true>;
    // [B][W + 4] input rows (sample x at 2 + x, 16-byte aligned, two zeros on
    // each side) in the FFT's own exchange buffer: they are read only by the
    // gather, which ends before the first exchange
    float2* srow = sm;
    const int WP = srow_pitch(W);
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int l0 = bx * B;
    const int l = l0 + f;

    // stage the block's B spectrum rows (W complex each)
    const int chunks = W >> 1;                         // two complex per 16 bytes
    if (threadIdx.x < 2 * B) {
        const int r = threadIdx.x >> 1;
        *reinterpret_cast<float4*>(srow + r * WP + ((threadIdx.x & 1) ? W + 2 : 0)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (BULK) {
        __shared__ uint64_t mbar;
        const uint32_t mb = smem_u32(&mbar);
        const int nrows = min(B, L - l0);              // >= 1: the grid covers rows 0 .. L-1
        if (threadIdx.x == 0) {
            mbar_init(mb, 1);
            mbar_arrive_expect_tx(mb, (uint32_t)(nrows * W * sizeof(float2)));
            for (int r = 0; r < nrows; ++r)
                bulk_g2s(srow + r * WP + 2, base + (size_t)(l0 + r) * N, (uint32_t)(W * sizeof(float2)), mb);
        }
        for (int r = nrows; r < B; ++r)                // rows past the end: zeros
            for (int c = threadIdx.x; c < chunks; c += fs_T(N) * B)
                *reinterpret_cast<float4*>(srow + r * WP + 2 + 2 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();                               // the mbarrier is initialised
        const bool ok = mbar_wait(mb, 0, wait);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && err) atomicOr(err, 2u);
            mbar_wait(mb, 0);                          // the copies in flight land first
            return false;
        }
    } else {
#pragma unroll
        for (int r = 0; r < B; ++r) {
            float2* dst = srow + r * WP + 2;
            const float2* src = base + (size_t)(l0 + r) * N;
            if (l0 + r < L) {
                for (int c = threadIdx.x; c < chunks; c += fs_T(N) * B) cp_async16(dst + 2 * c, src + 2 * c);
            } else {
                for (int c = threadIdx.x; c < chunks; c += fs_T(N) * B)
                    *reinterpret_cast<float4*>(dst + 2 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();

    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
    if (l >= 1 && l < L) {
        const float2* myrow = srow + f * WP + 2;
        const int den = 2 * l;
        const float inv = 1.f / (float)den;
        const int step = STEPX * Hp;
        const int sA = step / den, sB = step - sA * den;
        const int halfW = W >> 1;
        const float2 zero = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < G0; ++m) {
            const int i = t + m * T;
            const int num = (i - N / 2) * Hp;
            int qf = floor_div(num, den);
            int rem = num - qf * den;
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const float fr = (float)rem * inv;
                const int c0 = qf + halfW;
                float2 acc;
                if constexpr (INTERP == FT_INTERP_LINEAR) {
                    // taps c0, c0 + 1; outside 0 .. W-1 the padding's zeros
                    const int cc = min(max(c0, -2), W);
                    const bool ok = FT_IN(cc + 3, WP, FT_DBG_NVMT_GATHER) && FT_IN(cc + 2, WP, FT_DBG_NVMT_GATHER);
                    const float2 a0 = ok ? myrow[cc] : zero, a1 = ok ? myrow[cc + 1] : zero;
                    acc = make_float2(fmaf(fr, a1.x - a0.x, a0.x), fmaf(fr, a1.y - a0.y, a0.y));
                } else {
                    acc = zero;
#pragma unroll
                    for (int d = -1; d <= 2; ++d) {
                        const float2 a = (unsigned)(c0 + d) < (unsigned)W ? myrow[c0 + d] : zero;
                        const float w = keys_w(fr - (float)d);
                        acc.x = fmaf(w, a.x, acc.x);
                        acc.y = fmaf(w, a.y, acc.y);
                    }
                }
                v[m * R0 + q] = acc;
                rem += sB;
                qf += sA;
                if (rem >= den) { rem -= den; qf += 1; }
            }
        }
    }
    __syncthreads();                                   // the staged rows are dead from here
    // The centring factor (-1)^i of the gathered samples is a shift of the
    // transform by N/2: with Z the transform of the taps, the row gets
    // G[s] = (-1)^(s + N/2) Z[(s + N/2) mod N], i.e. Z[s'] (times (-1)^s') goes
    // to position (s' + N/2) mod N
    F::template run<0>(v, sm, t, f, stw);
    if (l >= L) return true;
    float2* row = base + (size_t)l * N;
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int s = F::out_pos(t, m, q);
            float2 val = v[m * RL + q];
            if (s & 1) val = make_float2(-val.x, -val.y);
            row[s < N / 2 ? s + N / 2 : s - N / 2] = val;
        }
    return true;
}
