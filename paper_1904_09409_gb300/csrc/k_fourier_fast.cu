// The band-limited (chirp-z) NVMT of Sec. IV fused with step 3, on the
// register-resident FFT of fft_fast.cuh: the same chain as k_fourier.cu (see
// there for the derivation),
//     row F (W) --F_W^- --> Fh --pre-chirp, 1/W--> y (M) --F_M^- --x Hc--> --F_M^+-->
//     z --post-chirp, 1/M, support mask, (-1)^k--> V (S) --F_S^+--> G, (-1)^(s+S/2)
// for W = S and M = 2W where all three lengths have a compile-time schedule.
//
// One block takes row l of B images (B = 256 / fs_T(M), at least 1): the four
// transforms of each image's row run in registers (B side by side, exchanging
// through one shared buffer), and the row's chirp tables (pre-chirp W + 1
// entries, post-chirp S, chirp spectrum M) are read once per block for its B
// images.  The grid runs the images fastest, so consecutive blocks share row l
// and its tables stay in L2: the tables are read from memory about once per
// call instead of once per image.  Between the transforms the data goes
// through shared memory once (the re-indexing u mod W, the change from the
// forward transform's output order to the inverse's input order, the
// truncation to S samples); threads that hold no transform of the shorter
// lengths W and S only join the barriers.
#include "fft_fast.cuh"

template <int W, int M, int S>
struct FrShape {
    static constexpr int TM = fs_T(M), TW = fs_T(W), TS = fs_T(S);
    static constexpr int B = TM >= 256 ? 1 : 256 / TM;         // rows (images) per block
    static constexpr int NT = TM * B;
    // resident blocks of NT threads per multiprocessor the registers are sized
    // for: four transforms in a row keep about 170 registers live unbounded;
    // 128 (two blocks of 256 threads) leaves at most a few words spilled
    static constexpr int MINB = 512 / NT > 0 ? 512 / NT : 1;
    static_assert(TW <= TM && TS <= TM, "the length-M transform has the most threads");
    static constexpr int SLOTS_W = FastFft<W, -1, B>::SLOTS, SLOTS_M = FastFft<M, -1, B>::SLOTS,
                         SLOTS_S = FastFft<S, -1, B>::SLOTS;
    static constexpr int SLOTS = SLOTS_M > SLOTS_W ? (SLOTS_M > SLOTS_S ? SLOTS_M : SLOTS_S)
                                                   : (SLOTS_W > SLOTS_S ? SLOTS_W : SLOTS_S);
};

template <int W, int M, int S>
__global__ void __launch_bounds__(FrShape<W, M, S>::NT, FrShape<W, M, S>::MINB)
k_nvmt_rows_fourier_fast(float2* __restrict__ ws, int Hp, int L, int batch, const float2* __restrict__ stw_w,
                         const float2* __restrict__ stw_m, const float2* __restrict__ stw_s,
                         const float2* __restrict__ chirp_u, const float2* __restrict__ chirp_x,
                         const float2* __restrict__ hc) {
    using Sh = FrShape<W, M, S>;
    constexpr int B = Sh::B, TW = Sh::TW, TS = Sh::TS;
    constexpr int EW = fs_E(W), EM = fs_E(M), ES = fs_E(S);
    using FW = FastFft<W, -1, B, true>;
    using FMf = FastFft<M, -1, B, true>;
    using FMi = FastFft<M, +1, B, true>;
    using FS = FastFft<S, +1, B, true>;
    constexpr int R0W = fs_radix(W, 0), G0W = EW / R0W, RLW = fs_radix(W, fs_nst(W) - 1), GLW = EW / RLW;
    constexpr int R0M = fs_radix(M, 0), G0M = EM / R0M, RLM = fs_radix(M, fs_nst(M) - 1), GLM = EM / RLM;
    constexpr int R0S = fs_radix(S, 0), G0S = ES / R0S, RLS = fs_radix(S, fs_nst(S) - 1), GLS = ES / RLS;
    extern __shared__ float2 sm[];
    const int l = blockIdx.y;
    const int f = threadIdx.x % B, t = threadIdx.x / B;
    const int img = blockIdx.x * B + f;
    const bool rowok = img < batch;
    float2* row = ws + ((size_t)img * L + l) * S;       // W values in, S values out
    if (l == 0) {                                       // the DC row is zero (the whole block)
        if (rowok)
            for (int k = t; k < S; k += Sh::TM) row[k] = make_float2(0.f, 0.f);
        return;
    }

    // ---- F_W^- of the row (threads t < TW)
    if (t < TW) {
        float2 v[EW];
#pragma unroll
        for (int m = 0; m < G0W; ++m)
#pragma unroll
            for (int q = 0; q < R0W; ++q)
                v[m * R0W + q] = rowok ? row[FW::template in_pos<0>(t, m, q)] : make_float2(0.f, 0.f);
        FW::template run<0>(v, sm, t, f, stw_w);
#pragma unroll
        for (int m = 0; m < GLW; ++m)
#pragma unroll
            for (int q = 0; q < RLW; ++q) sm[spos(FW::out_pos(t, m, q)) * B + f] = v[m * RLW + q];
    } else {
        FW::template idle<0>();
    }
    __syncthreads();

    // ---- y[i] = Fh[u mod W] (+-1/W, halved at u = +-W/2) x pre-chirp, u = i - W/2 (i <= W), 0 beyond
    float2 v[EM];
    {
        const float2* cu = chirp_u + (size_t)l * (W + 1);
        const float invW = 1.f / (float)W;
#pragma unroll
        for (int m = 0; m < G0M; ++m)
#pragma unroll
            for (int q = 0; q < R0M; ++q) {
                const int i = FMf::template in_pos<0>(t, m, q);
                float2 y = make_float2(0.f, 0.f);
                if (i <= W) {
                    const int u = i - W / 2;
                    const int k = u < 0 ? u + W : u;
                    float sc = (u & 1) ? -invW : invW;
                    if (u == W / 2 || u == -W / 2) sc *= 0.5f;
                    const float2 a = sm[spos(k) * B + f];
                    y = cmul(make_float2(a.x * sc, a.y * sc), __ldg(cu + i));
                }
                v[m * R0M + q] = y;
            }
    }
    __syncthreads();

    // ---- F_M^-, times the chirp spectrum, back to the input order, F_M^+
    FMf::template run<0>(v, sm, t, f, stw_m);
    {
        const float2* hl = hc + (size_t)l * M;
#pragma unroll
        for (int m = 0; m < GLM; ++m)
#pragma unroll
            for (int q = 0; q < RLM; ++q) {
                const int k = FMf::out_pos(t, m, q);
                sm[spos(k) * B + f] = cmul(v[m * RLM + q], __ldg(hl + k));
            }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < G0M; ++m)
#pragma unroll
        for (int q = 0; q < R0M; ++q) v[m * R0M + q] = sm[spos(FMi::template in_pos<0>(t, m, q)) * B + f];
    __syncthreads();
    FMi::template run<0>(v, sm, t, f, stw_m);

    // ---- V[k] = z[k] / M x post-chirp inside the support, (-1)^k, k < S
    {
        const float2* cx = chirp_x + (size_t)l * S;
        const float invM = 1.f / (float)M;
        const long long den = 2ll * l;
#pragma unroll
        for (int m = 0; m < GLM; ++m)
#pragma unroll
            for (int q = 0; q < RLM; ++q) {
                const int k = FMi::out_pos(t, m, q);
                if (k < S) {
                    const long long num = (long long)(k - S / 2) * Hp;       // p = num / den
                    float2 r = make_float2(0.f, 0.f);
                    if (num >= -(long long)(W / 2) * den && num <= (long long)(W / 2 - 1) * den) {
                        r = cmul(v[m * RLM + q], __ldg(cx + k));
                        const float sc = (k & 1) ? -invM : invM;
                        r = make_float2(r.x * sc, r.y * sc);
                    }
                    sm[spos(k) * B + f] = r;
                }
            }
    }
    __syncthreads();

    // ---- step 3: F_S^+ (threads t < TS), output sign (-1)^(s + S/2)
    if (t < TS) {
        float2 g[ES];
#pragma unroll
        for (int m = 0; m < G0S; ++m)
#pragma unroll
            for (int q = 0; q < R0S; ++q) g[m * R0S + q] = sm[spos(FS::template in_pos<0>(t, m, q)) * B + f];
        __syncthreads();
        FS::template run<0>(g, sm, t, f, stw_s);
        if (rowok) {
#pragma unroll
            for (int m = 0; m < GLS; ++m)
#pragma unroll
                for (int q = 0; q < RLS; ++q) {
                    const int s = FS::out_pos(t, m, q);
                    float2 val = g[m * RLS + q];
                    if ((s + S / 2) & 1) val = make_float2(-val.x, -val.y);
                    row[s] = val;
                }
        }
    } else {
        __syncthreads();
        FS::template idle<0>();
    }
}

// Transpose of the above (see k_nvmt_rows_fourier_adj in k_fourier.cu): with
// O the output sign, D_x the post-chirp / 1/M / mask / (-1)^k, D_h the chirp
// spectrum, D_u the pre-chirp and P the re-indexing u mod W with its weights,
//     gF = F_W^+ P^T conj(D_u) F_M^+ conj(D_h) F_M^- conj(D_x) F_S^- O gG.
template <int W, int M, int S>
__global__ void __launch_bounds__(FrShape<W, M, S>::NT, FrShape<W, M, S>::MINB)
k_nvmt_rows_fourier_adj_fast(float2* __restrict__ ws, int Hp, int L, int batch, const float2* __restrict__ stw_w,
                             const float2* __restrict__ stw_m, const float2* __restrict__ stw_s,
                             const float2* __restrict__ chirp_u, const float2* __restrict__ chirp_x,
                             const float2* __restrict__ hc) {
    using Sh = FrShape<W, M, S>;
    constexpr int B = Sh::B, TW = Sh::TW, TS = Sh::TS;
    constexpr int EW = fs_E(W), EM = fs_E(M), ES = fs_E(S);
    using FS = FastFft<S, -1, B, true>;
    using FMf = FastFft<M, -1, B, true>;
    using FMi = FastFft<M, +1, B, true>;
    using FW = FastFft<W, +1, B, true>;
    constexpr int R0W = fs_radix(W, 0), G0W = EW / R0W, RLW = fs_radix(W, fs_nst(W) - 1), GLW = EW / RLW;
    constexpr int R0M = fs_radix(M, 0), G0M = EM / R0M, RLM = fs_radix(M, fs_nst(M) - 1), GLM = EM / RLM;
    constexpr int R0S = fs_radix(S, 0), G0S = ES / R0S, RLS = fs_radix(S, fs_nst(S) - 1), GLS = ES / RLS;
    extern __shared__ float2 sm[];
    const int l = blockIdx.y;
    const int f = threadIdx.x % B, t = threadIdx.x / B;
    const int img = blockIdx.x * B + f;
    const bool rowok = img < batch;
    float2* row = ws + ((size_t)img * L + l) * S;       // S values in, W values out
    if (l == 0) {
        if (rowok)
            for (int x = t; x < W; x += Sh::TM) row[x] = make_float2(0.f, 0.f);
        return;
    }

    // ---- O, F_S^- (threads t < TS)
    if (t < TS) {
        float2 g[ES];
#pragma unroll
        for (int m = 0; m < G0S; ++m)
#pragma unroll
            for (int q = 0; q < R0S; ++q) {
                const int s = FS::template in_pos<0>(t, m, q);
                float2 val = rowok ? row[s] : make_float2(0.f, 0.f);
                if ((s + S / 2) & 1) val = make_float2(-val.x, -val.y);
                g[m * R0S + q] = val;
            }
        FS::template run<0>(g, sm, t, f, stw_s);
#pragma unroll
        for (int m = 0; m < GLS; ++m)
#pragma unroll
            for (int q = 0; q < RLS; ++q) sm[spos(FS::out_pos(t, m, q)) * B + f] = g[m * RLS + q];
    } else {
        FS::template idle<0>();
    }
    __syncthreads();

    // ---- conj(D_x) on k < S, zero beyond, F_M^-
    float2 v[EM];
    {
        const float2* cx = chirp_x + (size_t)l * S;
        const float invM = 1.f / (float)M;
        const long long den = 2ll * l;
#pragma unroll
        for (int m = 0; m < G0M; ++m)
#pragma unroll
            for (int q = 0; q < R0M; ++q) {
                const int k = FMf::template in_pos<0>(t, m, q);
                float2 r = make_float2(0.f, 0.f);
                if (k < S) {
                    const long long num = (long long)(k - S / 2) * Hp;
                    if (num >= -(long long)(W / 2) * den && num <= (long long)(W / 2 - 1) * den) {
                        const float2 c = __ldg(cx + k);
                        r = cmul(sm[spos(k) * B + f], make_float2(c.x, -c.y));
                        const float sc = (k & 1) ? -invM : invM;
                        r = make_float2(r.x * sc, r.y * sc);
                    }
                }
                v[m * R0M + q] = r;
            }
    }
    __syncthreads();
    FMf::template run<0>(v, sm, t, f, stw_m);
    {
        const float2* hl = hc + (size_t)l * M;
#pragma unroll
        for (int m = 0; m < GLM; ++m)
#pragma unroll
            for (int q = 0; q < RLM; ++q) {
                const int k = FMf::out_pos(t, m, q);
                const float2 h = __ldg(hl + k);
                sm[spos(k) * B + f] = cmul(v[m * RLM + q], make_float2(h.x, -h.y));
            }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < G0M; ++m)
#pragma unroll
        for (int q = 0; q < R0M; ++q) v[m * R0M + q] = sm[spos(FMi::template in_pos<0>(t, m, q)) * B + f];
    __syncthreads();
    FMi::template run<0>(v, sm, t, f, stw_m);
#pragma unroll
    for (int m = 0; m < GLM; ++m)
#pragma unroll
        for (int q = 0; q < RLM; ++q) {
            const int k = FMi::out_pos(t, m, q);
            if (k <= W) sm[spos(k) * B + f] = v[m * RLM + q];       // z[i], i = u + W/2 <= W
        }
    __syncthreads();

    // ---- conj(D_u) and P^T: index x collects u = x (x <= W/2) or x - W, and
    // index W/2 also u = -W/2; weight (-1)^u / W, halved at u = +-W/2; then F_W^+
    if (t < TW) {
        const float2* cu = chirp_u + (size_t)l * (W + 1);
        const float invW = 1.f / (float)W;
        float2 a[EW];
#pragma unroll
        for (int m = 0; m < G0W; ++m)
#pragma unroll
            for (int q = 0; q < R0W; ++q) {
                const int x = FW::template in_pos<0>(t, m, q);
                const int u = x <= W / 2 ? x : x - W;
                float sc = (u & 1) ? -invW : invW;
                if (x == W / 2) sc *= 0.5f;
                const int i = u + W / 2;
                const float2 c = __ldg(cu + i);
                float2 r = cmul(sm[spos(i) * B + f], make_float2(c.x, -c.y));
                r = make_float2(r.x * sc, r.y * sc);
                if (x == W / 2) {                       // u = -W/2, the same weight
                    const float2 c2 = __ldg(cu);
                    const float2 r2 = cmul(sm[f], make_float2(c2.x, -c2.y));
                    const float sc2 = ((-W / 2) & 1) ? -0.5f * invW : 0.5f * invW;
                    r = make_float2(r.x + r2.x * sc2, r.y + r2.y * sc2);
                }
                a[m * R0W + q] = r;
            }
        __syncthreads();
        FW::template run<0>(a, sm, t, f, stw_w);
        if (rowok) {
#pragma unroll
            for (int m = 0; m < GLW; ++m)
#pragma unroll
                for (int q = 0; q < RLW; ++q) row[FW::out_pos(t, m, q)] = a[m * RLW + q];
        }
    } else {
        __syncthreads();
        FW::template idle<0>();
    }
}

// ------------------------------------------------------------------ dispatch
#define FR_FAST_LENGTHS(X) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(2048)

bool fourier_fast_ok(int W, int M, int S) {
    if (W != S || M != 2 * W) return false;
    switch (W) {
#define X(n) case n:
        FR_FAST_LENGTHS(X)
#undef X
        return true;
    }
    return false;
}

template <int N>
static cudaError_t go_fourier(bool adj, float2* ws, int Hp, int L, int batch, const float2* stw_w,
                              const float2* stw_m, const float2* stw_s, const float2* cu, const float2* cx,
                              const float2* hc, cudaStream_t st) {
    using Sh = FrShape<N, 2 * N, N>;
    const size_t sm = (size_t)Sh::SLOTS * sizeof(float2);
    const dim3 grid((batch + Sh::B - 1) / Sh::B, L);
    cudaError_t e;
    if (adj) {
        e = cudaFuncSetAttribute(k_nvmt_rows_fourier_adj_fast<N, 2 * N, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_nvmt_rows_fourier_adj_fast<N, 2 * N, N><<<grid, Sh::NT, sm, st>>>(ws, Hp, L, batch, stw_w, stw_m, stw_s, cu,
                                                                           cx, hc);
    } else {
        e = cudaFuncSetAttribute(k_nvmt_rows_fourier_fast<N, 2 * N, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_nvmt_rows_fourier_fast<N, 2 * N, N><<<grid, Sh::NT, sm, st>>>(ws, Hp, L, batch, stw_w, stw_m, stw_s, cu, cx,
                                                                       hc);
    }
    return cudaGetLastError();
}

cudaError_t launch_nvmt_rows_fourier_fast(bool adjoint, float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                          const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                          const float2* chirp_x, const float2* hc, int batch, cudaStream_t st) {
    if (!fourier_fast_ok(W, fm.N, S) || !fw.stw || !fm.stw || !fs.stw) return cudaErrorNotSupported;
    switch (W) {
#define X(n) case n: return go_fourier<n>(adjoint, ws, Hp, L, batch, fw.stw, fm.stw, fs.stw, chirp_u, chirp_x, hc, st);
        FR_FAST_LENGTHS(X)
#undef X
    }
    return cudaErrorNotSupported;
}
