// Batched out-of-place transpose in[b][R][C] -> out[b][C][R] through 32 x 32
// shared-memory tiles (padded against bank conflicts).  The inverse (dual)
// funnel transform of Sec. 3.1 runs the regular transform on the transposed
// image (x and y exchange roles), and its adjoint transposes the gradient back.
#include "ft_internal.cuh"

#define TP_TILE 32
#define TP_ROWS 8

__global__ void __launch_bounds__(TP_TILE * TP_ROWS)
k_transpose(const float* __restrict__ in, float* __restrict__ out, int R, int C) {
    __shared__ float tile[TP_TILE][TP_TILE + 1];
    const size_t img = blockIdx.z;
    const float* src = in + img * (size_t)R * C;
    float* dst = out + img * (size_t)R * C;
    const int c0 = blockIdx.x * TP_TILE, r0 = blockIdx.y * TP_TILE;
    for (int j = threadIdx.y; j < TP_TILE; j += TP_ROWS) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[j][threadIdx.x] = src[(size_t)r * C + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < TP_TILE; j += TP_ROWS) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[(size_t)c * R + r] = tile[threadIdx.x][j];
    }
}

cudaError_t launch_transpose(const float* in, float* out, int R, int C, int batch, cudaStream_t st) {
    dim3 grid((C + TP_TILE - 1) / TP_TILE, (R + TP_TILE - 1) / TP_TILE, batch);
    k_transpose<<<grid, dim3(TP_TILE, TP_ROWS), 0, st>>>(in, out, R, C);
    return cudaGetLastError();
}
