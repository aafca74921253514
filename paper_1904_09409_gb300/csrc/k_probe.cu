// FP32 FMA throughput probe: the measurement behind the ALU roofline that the
// benchmark reports for its arithmetic-heavy legs (the band-limited
// interpolator, the tensor-core transforms' SIMT work).  Every thread runs
// FT_PROBE_CHAINS independent FMA chains (enough independent work to keep the
// pipe busy at full occupancy) for `iters` rounds and stores their sum, so no
// operation can be eliminated.  FLOPs of one call = blocks x 256 x iters x
// FT_PROBE_CHAINS x 2.
#include "ft_internal.cuh"

#define FT_PROBE_CHAINS 8

__global__ void __launch_bounds__(256) k_fma_probe(float* __restrict__ out, int iters, float a, float b) {
    float x[FT_PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < FT_PROBE_CHAINS; ++k) x[k] = (float)threadIdx.x * 1e-3f + (float)k;
#pragma unroll 16
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < FT_PROBE_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < FT_PROBE_CHAINS; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" ft_status ft_fma_probe(float* d_out, int blocks, int iters, void* stream) {
    if (!d_out || blocks < 1 || iters < 1) return FT_ERR_INVALID_ARG;
    k_fma_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_out, iters, 0.999999f, 1e-7f);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FT_OK : ft_record_cuda(e, "ft_fma_probe");
}
