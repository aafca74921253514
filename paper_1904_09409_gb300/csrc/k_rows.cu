// Row transforms of the funnel transform (one frequency row l per transform).
//
//  k_nvmt_rows          steps 2 and 3 (Sec. 3.1, eqs. 17-18): the NVMT
//                       x' = (w2 / w_max) x with w2 = 2 pi l / H', w_max = pi, i.e.
//                       sample x' (centred, x' in [-S/2, S/2)) reads the row at
//                       x = x' H' / (2 l), interpolated in 1D with the row zero
//                       outside the image columns; then the transform along x'
//                       with the exp(+j) kernel, G[m] = sum_x' V[x'] e^{+j 2 pi m x'/S}.
//                       Row l = 0 is set to zero (the NVMT is degenerate there).
//  k_nvmt_rows_adjoint  the transpose: gV[x'] = sum_m gG[m] e^{-j 2 pi m x'/S},
//                       then every column x gathers the weights of the samples x'
//                       whose interpolation taps touched it (deterministic; no
//                       atomics).
//
// The sample position is split exactly: x' H' = q (2 l) + rem with q = floor and
// 0 <= rem < 2 l in integer arithmetic; the fraction is the single correctly
// rounded FP32 division rem / (2 l).
//
// Centred indices: with i = x' + S/2 and s = m + S/2,
// e^{+j 2 pi m x'/S} = e^{+j 2 pi s i / S} (-1)^i (-1)^s (-1)^{S/2}, so the gather
// multiplies by (-1)^i and the store by (-1)^{s + S/2}; the transpose mirrors it.
//
// Each block owns RB whole rows of one image and rewrites them in place (the
// workspace row pitch is S >= W).
#include "ft_internal.cuh"

__global__ void __launch_bounds__(FT_THREADS)
k_nvmt_rows(float2* __restrict__ ws, int W, int S, int Hp, int L, int interp, FftLen fx,
            int logRB) {
    extern __shared__ float2 smem[];
    const int RB = 1 << logRB;
    float2* srow = smem;                       // [W][RB]
    float2* a = smem + (W << logRB);           // [S][RB]
    float2* b = a + (S << logRB);              // [S][RB]
    const int img = blockIdx.y;
    const int l0 = blockIdx.x * RB;
    float2* base = ws + (size_t)img * L * S;

    for (int idx = threadIdx.x; idx < (W << logRB); idx += blockDim.x) {
        const int x = idx % W;
        const int r = idx / W;
        const int l = l0 + r;
        srow[(x << logRB) + r] = (l < L) ? base[(size_t)l * S + x] : make_float2(0.f, 0.f);
    }
    __syncthreads();

    const int dlo = interp == FT_INTERP_LINEAR ? 0 : -1;
    const int dhi = interp == FT_INTERP_LINEAR ? 1 : 2;
    const int halfW = W >> 1;
    for (int idx = threadIdx.x; idx < (S << logRB); idx += blockDim.x) {
        const int r = idx & (RB - 1);
        const int i = idx >> logRB;
        const int l = l0 + r;
        float2 v = make_float2(0.f, 0.f);
        if (l >= 1 && l < L) {
            const int num = (i - (S >> 1)) * Hp;
            const int den = 2 * l;
            const int q = floor_div(num, den);
            const float fr = (float)(num - q * den) / (float)den;
            for (int d = dlo; d <= dhi; ++d) {
                const int col = q + d + halfW;
                if (col >= 0 && col < W) {
                    const float w = tap_weight(interp, d, fr);
                    const float2 s = srow[(col << logRB) + r];
                    v.x += w * s.x;
                    v.y += w * s.y;
                }
            }
            if (i & 1) v = make_float2(-v.x, -v.y);
        }
        a[(i << logRB) + r] = v;
    }
    __syncthreads();
    const float2* z = cta_fft<+1>(a, b, fx, logRB);

    const int sh = S >> 1;
    for (int idx = threadIdx.x; idx < (S << logRB); idx += blockDim.x) {
        const int s = idx % S;
        const int r = idx / S;
        const int l = l0 + r;
        if (l >= L) continue;
        float2 v = z[(s << logRB) + r];
        if ((s + sh) & 1) v = make_float2(-v.x, -v.y);
        base[(size_t)l * S + s] = v;
    }
}

__global__ void __launch_bounds__(FT_THREADS)
k_nvmt_rows_adjoint(float2* __restrict__ ws, int W, int S, int Hp, int L, int interp, FftLen fx,
                    int logRB) {
    extern __shared__ float2 smem[];
    const int RB = 1 << logRB;
    float2* a = smem;                          // [S][RB]
    float2* b = a + (S << logRB);              // [S][RB]
    const int img = blockIdx.y;
    const int l0 = blockIdx.x * RB;
    float2* base = ws + (size_t)img * L * S;

    for (int idx = threadIdx.x; idx < (S << logRB); idx += blockDim.x) {
        const int s = idx % S;
        const int r = idx / S;
        const int l = l0 + r;
        float2 v = (l < L) ? base[(size_t)l * S + s] : make_float2(0.f, 0.f);
        if (s & 1) v = make_float2(-v.x, -v.y);
        a[(s << logRB) + r] = v;
    }
    __syncthreads();
    const float2* z = cta_fft<-1>(a, b, fx, logRB);

    // gV[x'] = (-1)^{i + S/2} z[i] with i = x' + S/2, i.e. (-1)^{x'} z[i] (S even)
    const int dlo = interp == FT_INTERP_LINEAR ? 0 : -1;
    const int dhi = interp == FT_INTERP_LINEAR ? 1 : 2;
    const int halfW = W >> 1;
    const int sh = S >> 1;
    for (int idx = threadIdx.x; idx < (W << logRB); idx += blockDim.x) {
        const int x = idx % W;
        const int r = idx / W;
        const int l = l0 + r;
        if (l >= L) continue;
        float2 acc = make_float2(0.f, 0.f);
        if (l >= 1) {
            const int xc = x - halfW;
            const int den = 2 * l;
            for (int d = dlo; d <= dhi; ++d) {
                // the sample x' whose floor(x' H' / (2 l)) equals xc - d, if any
                const int q = xc - d;
                const int xp = ceil_div(q * den, Hp);
                const int num = xp * Hp;
                if (num >= (q + 1) * den || xp < -sh || xp >= sh) continue;
                const float fr = (float)(num - q * den) / (float)den;
                const float w = tap_weight(interp, d, fr);
                float2 g = z[((xp + sh) << logRB) + r];
                if (xp & 1) g = make_float2(-g.x, -g.y);
                acc.x += w * g.x;
                acc.y += w * g.y;
            }
        }
        base[(size_t)l * S + x] = acc;
    }
}

static size_t rows_smem(int W, int S, int logRB, bool fwd) {
    return (size_t)((fwd ? W : 0) + 2 * S) * ((size_t)1 << logRB) * sizeof(float2);
}

cudaError_t launch_nvmt_rows(float2* ws, int W, int S, int Hp, int L, int interp,
                             const FftLen& fx, int logRB, int batch, cudaStream_t st) {
    const size_t sm = rows_smem(W, S, logRB, true);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((L + (1 << logRB) - 1) >> logRB, batch);
    k_nvmt_rows<<<grid, FT_THREADS, sm, st>>>(ws, W, S, Hp, L, interp, fx, logRB);
    return cudaGetLastError();
}

cudaError_t launch_nvmt_rows_adjoint(float2* ws, int W, int S, int Hp, int L, int interp,
                                     const FftLen& fx, int logRB, int batch, cudaStream_t st) {
    const size_t sm = rows_smem(W, S, logRB, false);
    cudaError_t e = cudaFuncSetAttribute(k_nvmt_rows_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((L + (1 << logRB) - 1) >> logRB, batch);
    k_nvmt_rows_adjoint<<<grid, FT_THREADS, sm, st>>>(ws, W, S, Hp, L, interp, fx, logRB);
    return cudaGetLastError();
}
