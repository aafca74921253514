// Step 2 with the band-limited interpolator (Sec. IV adopts a chirp-z based 1D
// interpolation for the NVMT), fused with step 3.
//
// Row l of the half spectrum, F[x] for centred x in [-W/2, W/2), is the sample
// set of the trigonometric polynomial
//     T(p) = (1/W) sum_{u=-W/2}^{W/2} ' Fh[u] exp(+j 2 pi u p / W),
//     Fh[u] = sum_x F[x] exp(-j 2 pi u x / W),
// where ' halves the two Nyquist terms u = +-W/2 (together Fh[W/2] cos(pi p)).
// The NVMT needs T at p = x' a with a = H'/(2 l), x' = -S/2 .. S/2-1, and zero
// where p is outside [-W/2, W/2-1].  With b = a / W and
//     u x' = (u^2 + x'^2 - (x' - u)^2) / 2                (Bluestein)
//     T(x' a) = exp(j pi b x'^2) sum_u [a_u exp(j pi b u^2)] exp(-j pi b (x' - u)^2)
// the sum is a linear convolution of W + 1 terms with a chirp of S + W taps,
// done as a circular convolution of length M >= S + W by FFTs:
//     y[u + W/2] = a_u exp(j pi b u^2),  a_u = Fh[u] / W (halved at u = +-W/2)
//     z = IFFT_M( FFT_M(y) * Hc ),  Hc = FFT_M(h), h[j mod M] = exp(-j pi b (j + W/2 - S/2)^2)
//     V[k] = z[k] exp(j pi b x'^2), k = x' + S/2, masked to the support.
// The chirps are computed on the host in FP64 after an exact integer reduction
// of the phase (pi b d^2 = 2 pi (H' d^2 mod 4 l W) / (4 l W)), rounded once to
// FP32; Hc is transformed once per plan on the GPU.  Then step 3 as in the
// other row kernels: G[m] = sum_x' V[x'] exp(+j 2 pi m x' / S).
//
// One block per row; all transforms are the generic shared-memory Stockham FFT
// (lengths W, M, M, S).
#include "ft_internal.cuh"

#define FR_THREADS 256

// exp(-2 pi i t / N) tables of the three lengths are passed as FftLen
__global__ void __launch_bounds__(FR_THREADS)
k_nvmt_rows_fourier(float2* __restrict__ ws, int W, int S, int Hp, int L, int M, FftLen fw, FftLen fm,
                    FftLen fs, const float2* __restrict__ chirp_u, const float2* __restrict__ chirp_x,
                    const float2* __restrict__ hc) {
    extern __shared__ float2 smem[];
    const int l = blockIdx.x;
    float2* a = smem;
    float2* b = smem + M;
    float2* row = ws + (size_t)blockIdx.y * L * S + (size_t)l * S;
    if (l == 0) {
        for (int k = threadIdx.x; k < S; k += blockDim.x) row[k] = make_float2(0.f, 0.f);
        return;
    }
    // Fh[u] = (-1)^u FFT_W(F)[u mod W]  (x = c - W/2 centred)
    for (int c = threadIdx.x; c < W; c += blockDim.x) a[c] = row[c];
    __syncthreads();
    float2* fh = cta_fft<-1>(a, b, fw, 0);
    float2* y = (fh == a) ? b : a;                     // the other buffer
    const float2* cu = chirp_u + (size_t)l * (W + 1);
    const float invW = 1.f / (float)W;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (i <= W) {
            const int u = i - W / 2;
            float2 f = fh[((u % W) + W) % W];
            float s = ((u & 1) ? -invW : invW);
            if (u == W / 2 || u == -W / 2) s *= 0.5f;
            f = make_float2(f.x * s, f.y * s);
            v = cmul(f, __ldg(cu + i));
        }
        y[i] = v;
    }
    __syncthreads();
    float2* Y = cta_fft<-1>(y, fh, fm, 0);
    const float2* hl = hc + (size_t)l * M;
    float2* o = (Y == y) ? fh : y;
    for (int i = threadIdx.x; i < M; i += blockDim.x) Y[i] = cmul(Y[i], __ldg(hl + i));
    __syncthreads();
    float2* z = cta_fft<+1>(Y, o, fm, 0);
    float2* v = (z == Y) ? o : Y;
    // V[k] = z[k] / M * exp(j pi b x'^2) inside the support, then (-1)^k for the
    // centred transform of step 3
    const float2* cx = chirp_x + (size_t)l * S;
    const float invM = 1.f / (float)M;
    const long long den = 2ll * l;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        const long long num = (long long)(k - S / 2) * Hp;       // p = num / den
        float2 r = make_float2(0.f, 0.f);
        if (num >= -(long long)(W / 2) * den && num <= (long long)(W / 2 - 1) * den) {
            r = cmul(z[k], __ldg(cx + k));
            r = make_float2(r.x * invM, r.y * invM);
            if (k & 1) r = make_float2(-r.x, -r.y);
        }
        v[k] = r;
    }
    __syncthreads();
    float2* G = cta_fft<+1>(v, z, fs, 0);                // z is the free buffer now
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        float2 g = G[s];
        if ((s + S / 2) & 1) g = make_float2(-g.x, -g.y);
        row[s] = g;
    }
}

// Transpose of the above (the adjoint for the real inner product, as the other
// row adjoints): every linear stage in reverse order, each replaced by its
// conjugate transpose.  The forward row map is
//     G = O F_S^+ D_x F_M^+ D_h F_M^- D_u P F_W^- F
// (F_N^sign the unnormalised DFT of length N, D_x the post-chirp / 1/M / mask /
// (-1)^k diagonal, D_h the chirp spectrum, D_u the pre-chirp on the W + 1 used
// entries, P the re-indexing u mod W with the +-1/W (halved at u = +-W/2)
// weights, O the (-1)^{s + S/2} output sign), so with (F_N^sign)^H = F_N^-sign
//     gF = F_W^+ P^T conj(D_u) F_M^+ conj(D_h) F_M^- conj(D_x) F_S^- O gG.
// P^T adds the two Nyquist entries u = -W/2 and u = +W/2 into index W/2.  Row 0
// (zero in the forward) gets zero.  In place: the S values of a row in, its W
// gradient values out (the row's first W entries), one block per row.
__global__ void __launch_bounds__(FR_THREADS)
k_nvmt_rows_fourier_adj(float2* __restrict__ ws, int W, int S, int Hp, int L, int M, FftLen fw, FftLen fm,
                        FftLen fs, const float2* __restrict__ chirp_u, const float2* __restrict__ chirp_x,
                        const float2* __restrict__ hc) {
    extern __shared__ float2 smem[];
    const int l = blockIdx.x;
    float2* a = smem;
    float2* b = smem + M;
    float2* row = ws + (size_t)blockIdx.y * L * S + (size_t)l * S;
    if (l == 0) {
        for (int x = threadIdx.x; x < W; x += blockDim.x) row[x] = make_float2(0.f, 0.f);
        return;
    }
    // O, then F_S^-
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        float2 g = row[s];
        if ((s + S / 2) & 1) g = make_float2(-g.x, -g.y);
        a[s] = g;
    }
    __syncthreads();
    float2* gv = cta_fft<-1>(a, b, fs, 0);
    float2* y = (gv == a) ? b : a;
    // conj(D_x) on the first S entries, zero on the rest of the length M
    const float2* cx = chirp_x + (size_t)l * S;
    const float invM = 1.f / (float)M;
    const long long den = 2ll * l;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        float2 r = make_float2(0.f, 0.f);
        if (k < S) {
            const long long num = (long long)(k - S / 2) * Hp;
            if (num >= -(long long)(W / 2) * den && num <= (long long)(W / 2 - 1) * den) {
                const float2 c = __ldg(cx + k);
                r = cmul(gv[k], make_float2(c.x, -c.y));
                const float sc = (k & 1) ? -invM : invM;
                r = make_float2(r.x * sc, r.y * sc);
            }
        }
        y[k] = r;
    }
    __syncthreads();
    // F_M^-, conj(D_h), F_M^+
    float2* Y = cta_fft<-1>(y, gv, fm, 0);
    float2* o = (Y == y) ? gv : y;
    const float2* hl = hc + (size_t)l * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const float2 h = __ldg(hl + i);
        Y[i] = cmul(Y[i], make_float2(h.x, -h.y));
    }
    __syncthreads();
    float2* z = cta_fft<+1>(Y, o, fm, 0);
    float2* acc = (z == Y) ? o : Y;
    // conj(D_u) and P^T: index x collects u = x (x <= W/2) or u = x - W, and
    // index W/2 also u = -W/2; weight (-1)^u / W, halved at u = +-W/2
    const float2* cu = chirp_u + (size_t)l * (W + 1);
    const float invW = 1.f / (float)W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int u = x <= W / 2 ? x : x - W;
        float sc = (u & 1) ? -invW : invW;
        if (x == W / 2) sc *= 0.5f;
        const int i = u + W / 2;
        const float2 c = __ldg(cu + i);
        float2 r = cmul(z[i], make_float2(c.x, -c.y));
        r = make_float2(r.x * sc, r.y * sc);
        if (x == W / 2) {                               // u = -W/2, same weight (W/2 even or odd alike)
            const float2 c2 = __ldg(cu);
            const float2 r2 = cmul(z[0], make_float2(c2.x, -c2.y));
            const float sc2 = ((-W / 2) & 1) ? -0.5f * invW : 0.5f * invW;
            r = make_float2(r.x + r2.x * sc2, r.y + r2.y * sc2);
        }
        acc[x] = r;
    }
    __syncthreads();
    // F_W^+ into the row's first W entries
    float2* gF = cta_fft<+1>(acc, z, fw, 0);
    for (int x = threadIdx.x; x < W; x += blockDim.x) row[x] = gF[x];
}

// in-place transform of the L chirp rows (length M) at plan creation
__global__ void __launch_bounds__(FR_THREADS) k_chirp_fft(float2* __restrict__ hc, int M, FftLen fm) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + M;
    float2* rowp = hc + (size_t)blockIdx.x * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) a[i] = rowp[i];
    __syncthreads();
    float2* r = cta_fft<-1>(a, b, fm, 0);
    for (int i = threadIdx.x; i < M; i += blockDim.x) rowp[i] = r[i];
}

cudaError_t launch_chirp_fft(float2* hc, int L, const FftLen& fm, cudaStream_t st) {
    const size_t sm = (size_t)2 * fm.N * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_chirp_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_chirp_fft<<<L, FR_THREADS, sm, st>>>(hc, fm.N, fm);
    return cudaGetLastError();
}

cudaError_t launch_nvmt_rows_fourier_adj(float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                         const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                         const float2* chirp_x, const float2* hc, int batch, cudaStream_t st) {
    const int M = fm.N;
    const size_t sm = (size_t)2 * M * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_fourier_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(L, batch);
    k_nvmt_rows_fourier_adj<<<grid, FR_THREADS, sm, st>>>(ws, W, S, Hp, L, M, fw, fm, fs, chirp_u, chirp_x, hc);
    return cudaGetLastError();
}

cudaError_t launch_nvmt_rows_fourier(float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                     const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                     const float2* chirp_x, const float2* hc, int batch, cudaStream_t st) {
    const int M = fm.N;
    const size_t sm = (size_t)2 * M * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_fourier, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(L, batch);
    k_nvmt_rows_fourier<<<grid, FR_THREADS, sm, st>>>(ws, W, S, Hp, L, M, fw, fm, fs, chirp_u, chirp_x, hc);
    return cudaGetLastError();
}
