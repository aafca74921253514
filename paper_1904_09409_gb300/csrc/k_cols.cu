// Column transforms of the funnel transform.
//
//  k_col_r2c  step 1 (Sec. 3.1, eq. 16): for every image column x, the Fourier
//             transform along y of the zero-expanded column (Sec. 4.2), kept for
//             l = 0 .. H'/2 (the other half is the conjugate, Sec. 3.1).  Two real
//             columns a, b are packed as a + i b into one complex transform Z and
//             separated with A_l = (Z_l + conj Z_{N-l}) / 2,
//             B_l = (Z_l - conj Z_{N-l}) / (2i).
//             With end/mid scales (1/H', 2/H') the same kernel is the transpose of
//             step 4.
//  k_col_c2r  step 4 (eq. 19): the inverse transform along w2 of the Hermitian
//             half spectrum of every map column (end bins through their real
//             part).  Two columns A, B are packed as Z = A + i B over the full
//             length N (Z_{N-l} = conj A_l + i conj B_l) and one inverse complex
//             transform gives a + i b.  With mid scale 1/2 and no 1/N it is the
//             transpose of step 1.
//
// The y coordinate is centred in the paper (y = row - H'/2).  The centring adds
// the factor (-1)^l to step 1 and again to step 4; the two cancel because steps 2
// and 3 act on one frequency row at a time, so neither kernel applies it.
//
// Layout: transform f of the block holds its sample n at smem[n * B + f]
// (B transforms interleaved), so consecutive threads touch consecutive
// columns in global memory and consecutive words in shared memory.
#include "ft_internal.cuh"

__global__ void __launch_bounds__(FT_THREADS)
k_col_r2c(const float* __restrict__ in, int rows_in, int ncols, int in_pitch, size_t in_img,
          int row0, FftLen f, int logB, float2* __restrict__ out, int out_pitch, size_t out_img,
          float end_scale, float mid_scale) {
    extern __shared__ float2 smem[];
    const int B = 1 << logB;
    const int N = f.N;
    float2* a = smem;
    float2* b = smem + (N << logB);
    const int img = blockIdx.y;
    const int c0 = blockIdx.x * 2 * B;
    const float* src = in + (size_t)img * in_img;

    for (int idx = threadIdx.x; idx < (N << logB); idx += blockDim.x) {
        const int fi = idx & (B - 1);
        const int row = (idx >> logB) - row0;
        const int c = c0 + 2 * fi;
        float2 v = make_float2(0.f, 0.f);
        if (row >= 0 && row < rows_in && c < ncols)
            v = *reinterpret_cast<const float2*>(src + (size_t)row * in_pitch + c);
        a[idx] = v;
    }
    __syncthreads();
    const float2* z = cta_fft<-1>(a, b, f, logB);

    float2* dst = out + (size_t)img * out_img;
    const int half = N >> 1;
    for (int idx = threadIdx.x; idx < ((half + 1) << logB); idx += blockDim.x) {
        const int fi = idx & (B - 1);
        const int l = idx >> logB;
        const int c = c0 + 2 * fi;
        if (c >= ncols) continue;
        const float2 zl = z[(l << logB) + fi];
        const float2 zm = z[(((N - l) % N) << logB) + fi];
        const float s = (l == 0 || l == half) ? end_scale : mid_scale;
        float4 o;
        o.x = 0.5f * s * (zl.x + zm.x);
        o.y = 0.5f * s * (zl.y - zm.y);
        o.z = 0.5f * s * (zl.y + zm.y);
        o.w = -0.5f * s * (zl.x - zm.x);
        *reinterpret_cast<float4*>(dst + (size_t)l * out_pitch + c) = o;
    }
}

__global__ void __launch_bounds__(FT_THREADS)
k_col_c2r(const float2* __restrict__ in, int ncols, int in_pitch, size_t in_img, FftLen f,
          int logB, float mid_scale, float* __restrict__ out, int row0, int rows_out,
          int out_pitch, size_t out_img, float out_scale) {
    extern __shared__ float2 smem[];
    const int B = 1 << logB;
    const int N = f.N;
    float2* a = smem;
    float2* b = smem + (N << logB);
    const int img = blockIdx.y;
    const int c0 = blockIdx.x * 2 * B;
    const float2* src = in + (size_t)img * in_img;
    const int half = N >> 1;

    for (int idx = threadIdx.x; idx < ((half + 1) << logB); idx += blockDim.x) {
        const int fi = idx & (B - 1);
        const int l = idx >> logB;
        const int c = c0 + 2 * fi;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < ncols) v = *reinterpret_cast<const float4*>(src + (size_t)l * in_pitch + c);
        if (l == 0 || l == half) {
            a[(l << logB) + fi] = make_float2(v.x, v.z);          // Re A + i Re B
        } else {
            v.x *= mid_scale; v.y *= mid_scale; v.z *= mid_scale; v.w *= mid_scale;
            a[(l << logB) + fi] = make_float2(v.x - v.w, v.y + v.z);          // A + i B
            a[((N - l) << logB) + fi] = make_float2(v.x + v.w, v.z - v.y);    // conj A + i conj B
        }
    }
    __syncthreads();
    const float2* z = cta_fft<+1>(a, b, f, logB);

    float* dst = out + (size_t)img * out_img;
    for (int idx = threadIdx.x; idx < (rows_out << logB); idx += blockDim.x) {
        const int fi = idx & (B - 1);
        const int r = idx >> logB;
        const int c = c0 + 2 * fi;
        if (c >= ncols) continue;
        const float2 v = z[((row0 + r) << logB) + fi];
        *reinterpret_cast<float2*>(dst + (size_t)r * out_pitch + c) =
            make_float2(v.x * out_scale, v.y * out_scale);
    }
}

static size_t col_smem(int N, int logB) { return (size_t)2 * ((size_t)N << logB) * sizeof(float2); }

cudaError_t launch_col_r2c(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img,
                           int row0, const FftLen& f, int logB, float2* out, int out_pitch,
                           size_t out_img, float end_scale, float mid_scale, int batch,
                           cudaStream_t st) {
    const size_t sm = col_smem(f.N, logB);
    cudaError_t e = cudaFuncSetAttribute(k_col_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + (2 << logB) - 1) / (2 << logB), batch);
    k_col_r2c<<<grid, FT_THREADS, sm, st>>>(in, rows_in, ncols, in_pitch, in_img, row0, f, logB, out,
                                           out_pitch, out_img, end_scale, mid_scale);
    return cudaGetLastError();
}

cudaError_t launch_col_c2r(const float2* in, int ncols, int in_pitch, size_t in_img,
                           const FftLen& f, int logB, float mid_scale, float* out, int row0,
                           int rows_out, int out_pitch, size_t out_img, float out_scale,
                           int batch, cudaStream_t st) {
    const size_t sm = col_smem(f.N, logB);
    cudaError_t e = cudaFuncSetAttribute(k_col_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + (2 << logB) - 1) / (2 << logB), batch);
    k_col_c2r<<<grid, FT_THREADS, sm, st>>>(in, ncols, in_pitch, in_img, f, logB, mid_scale, out, row0,
                                           rows_out, out_pitch, out_img, out_scale);
    return cudaGetLastError();
}
