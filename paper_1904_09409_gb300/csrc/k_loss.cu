// Loss of the gradient workload on the parameter map: r = |P| * scale - T,
// per-image loss mean(r^2), and the gradient of the batch mean with respect to
// P, 2 r scale sign(P) / (batch * cells) (sign(0) = 0).  The paper fits nothing
// by gradient; this loss exists so that line parameters or upstream filters can
// be fitted through ft_backward, the exact adjoint of the transform.
//
// The per-image sums are deterministic: each of LOSS_BLOCKS blocks of an image
// reduces a fixed slice in a fixed order (FP32 with Kahan compensation per
// thread, then a tree) and writes one partial; a second kernel adds the
// partials of an image in index order.
#include "ft_internal.cuh"

#define LOSS_THREADS 256
#define LOSS_BLOCKS 64

__global__ void __launch_bounds__(LOSS_THREADS)
k_abs_mse_grad(const float* __restrict__ map, const float* __restrict__ target, size_t cells, float scale,
               float gscale, float* __restrict__ grad, float* __restrict__ partial) {
    __shared__ float red[LOSS_THREADS];
    const size_t img = blockIdx.y;
    const float* P = map + img * cells;
    const float* T = target + img * cells;
    float* G = grad + img * cells;
    float acc = 0.f, comp = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += stride) {
        const float p = P[i];
        const float r = fabsf(p) * scale - T[i];
        const float y = r * r - comp;               // Kahan summation
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
        const float sg = p > 0.f ? 1.f : (p < 0.f ? -1.f : 0.f);
        if (G) G[i] = 2.f * r * scale * sg * gscale;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[img * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_loss_finish(const float* __restrict__ partial, int nblk, size_t cells, float* __restrict__ loss) {
    const int img = blockIdx.x;
    float s = 0.f, comp = 0.f;
    for (int b = 0; b < nblk; ++b) {
        const float y = partial[(size_t)img * nblk + b] - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    loss[img] = s / (float)cells;
}

size_t loss_partial_bytes(int batch) { return (size_t)batch * LOSS_BLOCKS * sizeof(float); }

cudaError_t launch_loss_finish(const float* partial, int nblk, size_t cells, float* loss, int batch, cudaStream_t st) {
    k_loss_finish<<<batch, 1, 0, st>>>(partial, nblk, cells, loss);
    return cudaGetLastError();
}

cudaError_t launch_abs_mse_grad(const float* map, const float* target, int batch, size_t cells, float scale,
                                float* loss, float* grad, float* partial, cudaStream_t st) {
    dim3 g1(LOSS_BLOCKS, batch);
    const float gscale = (float)(1.0 / ((double)batch * (double)cells));
    k_abs_mse_grad<<<g1, LOSS_THREADS, 0, st>>>(map, target, cells, scale, gscale, grad, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss_finish<<<batch, 1, 0, st>>>(partial, LOSS_BLOCKS, cells, loss);
    return cudaGetLastError();
}
