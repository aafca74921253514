// Line verification of Sec. 4.5: for every peak of the detected list, the band
// of 2h + 1 pixels centred on the peak's candidate line is integrated along the
// line's length, and the resulting profile across the band decides whether the
// line exists.
//
// Geometry (regular space, eqs. 22-23): the cell (t, s) of an H' x S map gives
// m = s - S/2, n = t - H'/2 and the line y = (2m/S) x + n in the centred
// coordinates of the expanded image; in the image's own rows and columns its
// centre row at column u is
//     v_c(u) = m (2u - W) / S + t - top,   top = (H' - H) / 2,
// taken as an exact integer floor and remainder.  The band samples rows
// v_c(u) + d, d = -h .. h, by linear interpolation between the two nearest rows;
// a sample counts only where both rows lie inside the image.  An inverse-space
// peak (eqs. 24-25) is the regular-space peak of the transposed image: the same
// arithmetic with rows and columns exchanged, done here through the strides.
// profile[d] = mean of the valid samples at offset d, length = valid samples on
// the centre line, and the line exists iff length >= min_length and
//     max(|p[0] - (p[-h] + p[h]) / 2|, |p[h] - p[-h]| / 2) >= min_contrast
// (a ridge raises the centre over both borders, a step edge separates them).
//
// One warp per peak: the lanes walk the band's length, then reduce.
#include "ft_internal.cuh"

#define FV_THREADS 256
#define FV_MAXH 3

__global__ void __launch_bounds__(FV_THREADS)
k_verify(const float* __restrict__ img, int H, int W, int stride_v, int stride_u, size_t img_stride, int S,
         int Hp, const ft_peak* __restrict__ peaks, const int32_t* __restrict__ count, int batch, int top_k, int h,
         float min_contrast, int min_length, float* __restrict__ profile, int32_t* __restrict__ length,
         int32_t* __restrict__ verdict) {
    const int gw = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (gw >= batch * top_k) return;                   // whole warps
    const int b = gw / top_k, j = gw - b * top_k;
    const int nb = 2 * h + 1;
    float* prof = profile + (size_t)gw * nb;
    if (j >= count[b]) {                               // beyond the detected list
        if (lane < nb) prof[lane] = 0.f;
        if (lane == 0) {
            length[gw] = 0;
            verdict[gw] = -1;
        }
        return;
    }
    const ft_peak p = peaks[gw];
    const int m = p.s - S / 2;
    const int c0 = p.t - (Hp - H) / 2;                 // t - top
    const float* im = img + (size_t)b * img_stride;
    float sum[2 * FV_MAXH + 1];
    int cnt[2 * FV_MAXH + 1];
#pragma unroll
    for (int d = 0; d < 2 * FV_MAXH + 1; ++d) {
        sum[d] = 0.f;
        cnt[d] = 0;
    }
    for (int u = lane; u < W; u += 32) {
        const int num = m * (2 * u - W);
        const int q = floor_div(num, S);
        const float fr = (float)(num - q * S) / (float)S;
        const int vc = q + c0;
        const float* col = im + (size_t)u * stride_u;
#pragma unroll
        for (int d = 0; d < 2 * FV_MAXH + 1; ++d) {
            if (d >= nb) break;
            const int v0 = vc + d - h;
            if (v0 >= 0 && v0 + 1 <= H - 1) {
                const float a0 = __ldg(col + (size_t)v0 * stride_v);
                const float a1 = __ldg(col + (size_t)(v0 + 1) * stride_v);
                sum[d] += fmaf(fr, a1 - a0, a0);
                cnt[d] += 1;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 2 * FV_MAXH + 1; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum[d] += __shfl_xor_sync(0xffffffffu, sum[d], o);
            cnt[d] += __shfl_xor_sync(0xffffffffu, cnt[d], o);
        }
    }
    if (lane == 0) {
        float pr[2 * FV_MAXH + 1];
#pragma unroll
        for (int d = 0; d < 2 * FV_MAXH + 1; ++d) {
            pr[d] = cnt[d] > 0 ? sum[d] / (float)cnt[d] : 0.f;
            if (d < nb) prof[d] = pr[d];
        }
        const float ridge = fabsf(pr[h] - 0.5f * (pr[0] + pr[2 * h]));
        const float step = 0.5f * fabsf(pr[2 * h] - pr[0]);
        length[gw] = cnt[h];
        verdict[gw] = (cnt[h] >= min_length && fmaxf(ridge, step) >= min_contrast) ? 1 : 0;
    }
}

cudaError_t launch_verify(const float* img, int H, int W, int stride_v, int stride_u, size_t img_stride, int S,
                          int Hp, const ft_peak* peaks, const int32_t* count, int batch, int top_k, int h,
                          float min_contrast, int min_length, float* profile, int32_t* length, int32_t* verdict,
                          cudaStream_t st) {
    if (h < 1 || h > FV_MAXH) return cudaErrorInvalidValue;
    const size_t threads = (size_t)batch * top_k * 32;
    const unsigned blocks = (unsigned)((threads + FV_THREADS - 1) / FV_THREADS);
    if (blocks == 0) return cudaSuccess;
    k_verify<<<blocks, FV_THREADS, 0, st>>>(img, H, W, stride_v, stride_u, img_stride, S, Hp, peaks, count, batch,
                                            top_k, h, min_contrast, min_length, profile, length, verdict);
    return cudaGetLastError();
}
