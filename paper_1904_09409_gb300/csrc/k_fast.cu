// Fixed-length versions of the column and row kernels (see k_cols.cu and
// k_rows.cu for what each step computes) built on the register-resident FFT of
// fft_fast.cuh.  Differences from the generic kernels:
//  * the column kernel reads its first pass directly from global memory; the
//    other two stage their inputs into shared memory with 16-byte cp.async
//    copies, all in flight at once (C2R: the Hermitian half, each row read once
//    for both n and N - n; rows: the B spectrum rows feeding the NVMT gather);
//    the last pass writes global memory directly where the output order allows;
//  * the NVMT sample x' H' / (2 l) of successive elements of a thread is stepped
//    exactly by adding the precomputed quotient and remainder of
//    (N / R0) H' / (2 l), so the inner loop has no integer division;
//  * the interpolation fraction is remainder * (1 / (2 l)) in FP32 (within one
//    rounding of the exact fraction).
#include "fft_fast.cuh"

// The last pass of the column R2C and the split of each complex transform (two
// real columns a + i b) into the two half spectra:
//     A[l] = (Z[l] + conj Z[N-l]) / 2,  B[l] = (Z[l] - conj Z[N-l]) / (2 i),
// scaled by end_scale (l = 0, N/2) or mid_scale, written as one float4 per row.
template <int N>
__device__ __forceinline__ void r2c_finish(float2 (&v)[fs_E(N)], float2* sm, int t, int f, const float2* stw,
                                           bool colok, float2* dst, int out_pitch, float end_scale,
                                           float mid_scale) {
    constexpr int B = fs_Bcol(N), E = fs_E(N), T = N / E;
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
            if (m + GL * q >= E / 2) sm[spos(F::out_pos(t, m, q)) * B + f] = v[m * RL + q];
    __syncthreads();
    if (!colok) return;
    auto el = [&](int j) -> float2 { return v[(j % GL) * RL + j / GL]; };
    auto split_z = [&](int l, float2 zl, float2 zm, float s) {
        float4 o;
        o.x = 0.5f * s * (zl.x + zm.x);
        o.y = 0.5f * s * (zl.y - zm.y);
        o.z = 0.5f * s * (zl.y + zm.y);
        o.w = -0.5f * s * (zl.x - zm.x);
        *reinterpret_cast<float4*>(dst + (size_t)l * out_pitch) = o;
    };
    // only t = 0 meets the end bins 0 and N/2 (N/2 is a multiple of T)
    if (t != 0) {
#pragma unroll
        for (int j = 0; j < E / 2; ++j)
            split_z(t + T * j, el(j), sm[spos(N - t - T * j) * B + f], mid_scale);
    } else {
        split_z(0, el(0), el(0), end_scale);
#pragma unroll
        for (int j = 1; j < E / 2; ++j) split_z(T * j, el(j), el(E - j), mid_scale);
        split_z(N / 2, el(E / 2), el(E / 2), end_scale);
    }
}

// The column kernel reads its first pass straight from global memory (8-byte
// loads of its column pair): staging the image tile through shared memory first
// measured slower on GB300 (67 vs 60 us for 32 images of 1024^2).
template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bcol(N), 1024 / (fs_T(N) * fs_Bcol(N)))
k_col_r2c_fast(const float* __restrict__ in, int rows_in, int ncols, int in_pitch, size_t in_img,
               int row0, const float2* __restrict__ stw, float2* __restrict__ out, int out_pitch,
               size_t out_img, float end_scale, float mid_scale) {
    constexpr int B = fs_Bcol(N), E = fs_E(N);
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    using F = FastFft<N, -1, B>;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = blockIdx.x * 2 * B + 2 * f;
    const bool colok = c < ncols;
    const float* src = in + (size_t)blockIdx.y * in_img + c;

    float2 v[E];
    if (colok && row0 == 0 && rows_in == N) {          // every row is an image row
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q)
                v[m * R0 + q] = __ldg(reinterpret_cast<const float2*>(
                    src + (size_t)F::template in_pos<0>(t, m, q) * in_pitch));
    } else {
#pragma unroll
        for (int m = 0; m < G0; ++m)
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                const int row = F::template in_pos<0>(t, m, q) - row0;
                float2 x = make_float2(0.f, 0.f);
                if (colok && row >= 0 && row < rows_in)
                    x = __ldg(reinterpret_cast<const float2*>(src + (size_t)row * in_pitch));
                v[m * R0 + q] = x;
            }
    }
    r2c_finish<N>(v, sm, t, f, stw, colok, out + (size_t)blockIdx.y * out_img + c, out_pitch, end_scale, mid_scale);
}

template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bc2r(N), 1024 / (fs_T(N) * fs_Bc2r(N)))
k_col_c2r_fast(const float2* __restrict__ in, int ncols, int in_pitch, size_t in_img,
               const float2* __restrict__ stw, float mid_scale, float* __restrict__ out, int row0,
               int rows_out, int out_pitch, size_t out_img, float out_scale, unsigned* __restrict__ tmax) {
    constexpr int B = fs_Bc2r(N), E = fs_E(N);
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    using F = FastFft<N, +1, B>;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = blockIdx.x * 2 * B + 2 * f;
    const bool colok = c < ncols;

    // stage the Hermitian half (rows 0 .. N/2, 2B complex each) with 16-byte async
    // copies; every row is read once and serves both n and N - n.  Thread (t, f)
    // copies the column pair f of rows t, t + T, ...
    float2* stg = sm;                                  // [N/2 + 1][2B]
    {
        const float2* src = in + (size_t)blockIdx.y * in_img + c + (size_t)t * in_pitch;
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
            float4 g = *reinterpret_cast<const float4*>(stg + (up ? n : N - n) * 2 * B + 2 * f);
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
        // j = m + GL q, of its column pair.  A tile is RS = c2r_tile_rows(N)
        // consecutive rows of one band (rows T j + RS u .. T j + RS u + RS - 1,
        // u < T / RS) of the block's 2B columns, 256 cells held by the RS B
        // consecutive threads t = RS u .. RS u + RS - 1.  Each thread puts
        // max(|re|, |im|) of its element of band j (the stored, scaled values;
        // NaN counts as 0, like a cell that is never a peak) at bm[j][thread] in
        // the exchange buffer, which the FFT no longer reads; then every warp
        // reduces tiles w, w + warps, ...: 4 conflict-free words per lane and
        // one redux.sync.
        constexpr int NT = fs_T(N) * B;                // threads of the block
        constexpr int RS = c2r_tile_rows(N), TPB = fs_T(N) / RS;   // tile rows, tiles per band
        static_assert(RS * B == 128, "a tile is 128 threads' values");
        static_assert(E * NT <= FastFft<N, +1, B>::SLOTS * 2, "band maxima fit the exchange buffer");
        unsigned* bm = reinterpret_cast<unsigned*>(sm);
#pragma unroll
        for (int m = 0; m < GL; ++m)
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const float a = fabsf(v[m * RL + q].x * out_scale), b = fabsf(v[m * RL + q].y * out_scale);
                bm[(m + GL * q) * NT + threadIdx.x] = colok ? __float_as_uint(fmaxf(fmaxf(a, b), 0.f)) : 0u;
            }
        __syncthreads();
        const int lane = threadIdx.x & 31;
        for (int w = threadIdx.x >> 5; w < E * TPB; w += NT / 32) {
            const int j = w / TPB, u = w - j * TPB;
            const unsigned* src = bm + j * NT + u * 128 + lane;
            unsigned x = max(max(src[0], src[32]), max(src[64], src[96]));
            x = __reduce_max_sync(0xffffffffu, x);
            if (lane == 0) tmax[((size_t)blockIdx.y * E * TPB + w) * gridDim.x + blockIdx.x] = x;
        }
    }
    if (!colok) return;
    // row n of the result goes to output row n - row0 when that is in range
    float* dst = out + (size_t)blockIdx.y * out_img + c;
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int rr = F::out_pos(t, m, q) - row0;
            if ((unsigned)rr < (unsigned)rows_out)
                *reinterpret_cast<float2*>(dst + (size_t)rr * out_pitch) =
                    make_float2(v[m * RL + q].x * out_scale, v[m * RL + q].y * out_scale);
        }
}

// The adjoint of step 4 fed straight from the loss of the gradient workload:
// the input column pair is not a stored gradient map but
//     g = 2 r scale sign(P) gscale,   r = |P| scale - T
// computed from the map P and the target T as the columns are loaded (the loss
// gradient of k_loss.cu), while every thread adds r^2 of its samples (FP32,
// compensated) and the block writes one partial of the image's loss.  Each map
// cell is loaded by exactly one thread, so the partials of an image's blocks
// add up to its sum of r^2.  Everything after the load is r2c_finish.
template <int N>
__global__ void __launch_bounds__(fs_T(N) * fs_Bcol(N), 1024 / (fs_T(N) * fs_Bcol(N)))
k_col_r2c_loss_fast(const float* __restrict__ map, const float* __restrict__ target, int ncols, size_t img_cells,
                    const float2* __restrict__ stw, float2* __restrict__ out, int out_pitch, size_t out_img,
                    float end_scale, float mid_scale, float scale, float gscale, float* __restrict__ partial) {
    constexpr int B = fs_Bcol(N), E = fs_E(N);
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    using F = FastFft<N, -1, B>;
    extern __shared__ float2 sm[];
    __shared__ float red[fs_T(N) * fs_Bcol(N)];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int c = blockIdx.x * 2 * B + 2 * f;
    const bool colok = c < ncols;
    const float* P = map + (size_t)blockIdx.y * img_cells + c;
    const float* Tg = target + (size_t)blockIdx.y * img_cells + c;

    float2 v[E];
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
                const float2 p = __ldg(reinterpret_cast<const float2*>(P + (size_t)row * ncols));
                const float2 tt = __ldg(reinterpret_cast<const float2*>(Tg + (size_t)row * ncols));
                const float r0 = fabsf(p.x) * scale - tt.x, r1 = fabsf(p.y) * scale - tt.y;
                add(r0 * r0);
                add(r1 * r1);
                const float s0 = p.x > 0.f ? 1.f : (p.x < 0.f ? -1.f : 0.f);
                const float s1 = p.y > 0.f ? 1.f : (p.y < 0.f ? -1.f : 0.f);
                g = make_float2(2.f * r0 * scale * s0 * gscale, 2.f * r1 * scale * s1 * gscale);
            }
            v[m * R0 + q] = g;
        }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = (fs_T(N) * fs_Bcol(N)) / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    r2c_finish<N>(v, sm, t, f, stw, colok, out + (size_t)blockIdx.y * out_img + c, out_pitch, end_scale, mid_scale);
}

// row pitch (complex) of the staged spectrum rows: W samples between two zero
// samples on each side (so a clamped tap index needs no bounds test); W + 4
// keeps 16-byte alignment for cp.async and shifts successive rows by 8 banks
__host__ __device__ constexpr int srow_pitch(int W) { return W + 4; }

// at most 64 registers, so that 4 blocks of 256 threads share a multiprocessor
template <int N, int INTERP>
__global__ void __launch_bounds__(fs_T(N) * fs_Brow(N), 1024 / (fs_T(N) * fs_Brow(N)))
k_nvmt_rows_fast(float2* __restrict__ ws, int W, int Hp, int L, const float2* __restrict__ stw) {
    constexpr int B = fs_Brow(N), E = fs_E(N), T = N / E;
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    constexpr int STEPX = N / R0;                      // x' distance between a thread's elements
    using F = FastFft<N, +1, B>;
    extern __shared__ float2 sm[];
    // [B][W + 4] input rows (sample x at 2 + x, 16-byte aligned, two zeros on
    // each side) in the FFT's own exchange buffer: they are read only by the
    // gather, which ends before the first exchange
    float2* srow = sm;
    const int WP = srow_pitch(W);
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int l0 = blockIdx.x * B;
    const int l = l0 + f;
    float2* base = ws + (size_t)blockIdx.y * L * N;

    // stage the block's B spectrum rows (W complex each) with 16-byte async copies
    const int chunks = W >> 1;                         // two complex per 16 bytes
    if (threadIdx.x < 2 * B) {
        const int r = threadIdx.x >> 1;
        *reinterpret_cast<float4*>(srow + r * WP + ((threadIdx.x & 1) ? W + 2 : 0)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
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
                    const float2 a0 = myrow[cc], a1 = myrow[cc + 1];
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
                if ((i + q * STEPX) & 1) acc = make_float2(-acc.x, -acc.y);
                v[m * R0 + q] = acc;
                rem += sB;
                qf += sA;
                if (rem >= den) { rem -= den; qf += 1; }
            }
        }
    }
    __syncthreads();                                   // the staged rows are dead from here
    F::template run<0>(v, sm, t, f, stw);
    if (l >= L) return;
    float2* row = base + (size_t)l * N;
#pragma unroll
    for (int m = 0; m < GL; ++m)
#pragma unroll
        for (int q = 0; q < RL; ++q) {
            const int s = F::out_pos(t, m, q);
            float2 val = v[m * RL + q];
            if ((s + N / 2) & 1) val = make_float2(-val.x, -val.y);
            row[s] = val;
        }
}

template <int N, int INTERP>
__global__ void __launch_bounds__(fs_T(N) * fs_Brow(N), 1024 / (fs_T(N) * fs_Brow(N)))
k_nvmt_rows_adjoint_fast(float2* __restrict__ ws, int W, int Hp, int L, const float2* __restrict__ stw) {
    constexpr int B = fs_Brow(N), E = fs_E(N), T = N / E;
    constexpr int R0 = fs_radix(N, 0), G0 = E / R0;
    constexpr int RL = fs_radix(N, fs_nst(N) - 1), GL = E / RL;
    using F = FastFft<N, -1, B>;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int l = blockIdx.x * B + f;
    float2* row = ws + (size_t)blockIdx.y * L * N + (size_t)l * N;

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
                if (rem[j] > lim && xp[j] >= -N / 2 && xp[j] < N / 2) {
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

// ------------------------------------------------------------------ dispatch
#define FT_FAST_LENGTHS(X) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192) X(192) X(384) X(768) X(1536)

template <int N>
static cudaError_t go_r2c(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img, int row0,
                          const float2* stw, float2* out, int out_pitch, size_t out_img, float es, float ms,
                          int batch, cudaStream_t st) {
    constexpr int B = fs_Bcol(N);
    const size_t sm = (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_r2c_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    k_col_r2c_fast<N><<<grid, fs_T(N) * B, sm, st>>>(in, rows_in, ncols, in_pitch, in_img, row0, stw, out,
                                                     out_pitch, out_img, es, ms);
    return cudaGetLastError();
}

template <int N>
static cudaError_t go_r2c_loss(const float* map, const float* target, int ncols, const float2* stw, float2* out,
                               int out_pitch, size_t out_img, float es, float ms, float scale, float gscale,
                               float* partial, int batch, cudaStream_t st) {
    constexpr int B = fs_Bcol(N);
    const size_t sm = (size_t)FastFft<N, -1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_r2c_loss_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    k_col_r2c_loss_fast<N><<<grid, fs_T(N) * B, sm, st>>>(map, target, ncols, (size_t)N * ncols, stw, out, out_pitch,
                                                          out_img, es, ms, scale, gscale, partial);
    return cudaGetLastError();
}

template <int N>
static cudaError_t go_c2r(const float2* in, int ncols, int in_pitch, size_t in_img, const float2* stw,
                          float mid, float* out, int row0, int rows_out, int out_pitch, size_t out_img,
                          float os, unsigned* tmax, int batch, cudaStream_t st) {
    constexpr int B = fs_Bc2r(N);
    const size_t sm = (size_t)FastFft<N, +1, B>::SLOTS * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_col_c2r_fast<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + 2 * B - 1) / (2 * B), batch);
    k_col_c2r_fast<N><<<grid, fs_T(N) * B, sm, st>>>(in, ncols, in_pitch, in_img, stw, mid, out, row0,
                                                     rows_out, out_pitch, out_img, os, tmax);
    return cudaGetLastError();
}

template <int N, int INTERP>
static cudaError_t go_rows_i(float2* ws, int W, int Hp, int L, const float2* stw, int batch, cudaStream_t st) {
    constexpr int B = fs_Brow(N);
    const size_t slots = FastFft<N, +1, B>::SLOTS, rows = (size_t)srow_pitch(W) * B;
    const size_t sm = (slots > rows ? slots : rows) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_fast<N, INTERP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((L + B - 1) / B, batch);
    k_nvmt_rows_fast<N, INTERP><<<grid, fs_T(N) * B, sm, st>>>(ws, W, Hp, L, stw);
    return cudaGetLastError();
}

template <int N>
static cudaError_t go_rows(float2* ws, int W, int Hp, int L, int interp, const float2* stw, int batch,
                           cudaStream_t st) {
    return interp == FT_INTERP_LINEAR ? go_rows_i<N, FT_INTERP_LINEAR>(ws, W, Hp, L, stw, batch, st)
                                      : go_rows_i<N, FT_INTERP_CUBIC>(ws, W, Hp, L, stw, batch, st);
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
                                float end_scale, float mid_scale, int batch, cudaStream_t st) {
    switch (f.N) {
#define X(n) case n: return go_r2c<n>(in, rows_in, ncols, in_pitch, in_img, row0, f.stw, out, out_pitch, \
                                      out_img, end_scale, mid_scale, batch, st);
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
                                     float scale, float gscale, float* partial, int batch, cudaStream_t st) {
    if (ncols & 1) return cudaErrorInvalidValue;
    switch (f.N) {
#define X(n) case n: return go_r2c_loss<n>(map, target, ncols, f.stw, out, out_pitch, out_img, end_scale, mid_scale, \
                                           scale, gscale, partial, batch, st);
        FT_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_col_c2r_fast(const float2* in, int ncols, int in_pitch, size_t in_img,
                                const FftLen& f, float mid_scale, float* out, int row0, int rows_out,
                                int out_pitch, size_t out_img, float out_scale, int batch,
                                cudaStream_t st, unsigned* tmax) {
    if (tmax && (row0 != 0 || rows_out != f.N)) return cudaErrorInvalidValue;
    switch (f.N) {
#define X(n) case n: return go_c2r<n>(in, ncols, in_pitch, in_img, f.stw, mid_scale, out, row0, rows_out, \
                                      out_pitch, out_img, out_scale, tmax, batch, st);
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
                                  int batch, cudaStream_t st) {
    switch (fx.N) {
#define X(n) case n: return go_rows<n>(ws, W, Hp, L, interp, fx.stw, batch, st);
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
