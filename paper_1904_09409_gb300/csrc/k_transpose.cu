// Batched out-of-place transpose in[b][R][C] -> out[b][C][R] through padded
// shared-memory tiles.  The inverse (dual)
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

// The same with 64 x 64 tiles for even R and C: every thread moves 8 float2
// (two adjacent columns of 8 rows in, two adjacent rows of 8 columns out), all
// loads of a thread in flight before its first store.
#define TP2_TILE 64
#define TP2_ROWS 8

__global__ void __launch_bounds__(32 * TP2_ROWS)
k_transpose64(const float* __restrict__ in, float* __restrict__ out, int R, int C) {
    __shared__ float tile[TP2_TILE][TP2_TILE + 1];
    const size_t img = blockIdx.z;
    const float* src = in + img * (size_t)R * C;
    float* dst = out + img * (size_t)R * C;
    const int c0 = blockIdx.x * TP2_TILE, r0 = blockIdx.y * TP2_TILE;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float2 v[TP2_TILE / TP2_ROWS];
#pragma unroll
    for (int k = 0; k < TP2_TILE / TP2_ROWS; ++k) {
        const int r = r0 + ty + TP2_ROWS * k, c = c0 + 2 * tx;
        v[k] = (r < R && c < C) ? __ldg(reinterpret_cast<const float2*>(src + (size_t)r * C + c))
                                : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < TP2_TILE / TP2_ROWS; ++k) {
        tile[ty + TP2_ROWS * k][2 * tx] = v[k].x;
        tile[ty + TP2_ROWS * k][2 * tx + 1] = v[k].y;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TP2_TILE / TP2_ROWS; ++k) {
        const int c = c0 + ty + TP2_ROWS * k, r = r0 + 2 * tx;
        if (c < C && r < R)
            *reinterpret_cast<float2*>(dst + (size_t)c * R + r) =
                make_float2(tile[2 * tx][ty + TP2_ROWS * k], tile[2 * tx + 1][ty + TP2_ROWS * k]);
    }
}

cudaError_t launch_transpose(const float* in, float* out, int R, int C, int batch, cudaStream_t st) {
    if (((R | C) & 1) == 0) {
        dim3 grid((C + TP2_TILE - 1) / TP2_TILE, (R + TP2_TILE - 1) / TP2_TILE, batch);
        k_transpose64<<<grid, dim3(32, TP2_ROWS), 0, st>>>(in, out, R, C);
        return cudaGetLastError();
    }
    dim3 grid((C + TP_TILE - 1) / TP_TILE, (R + TP_TILE - 1) / TP_TILE, batch);
    k_transpose<<<grid, dim3(TP_TILE, TP_ROWS), 0, st>>>(in, out, R, C);
    return cudaGetLastError();
}
