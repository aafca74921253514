// Peak detection of Sec. 4.4 on the brightness |P| of each map.
//
// The paper visits the cells in order of decreasing brightness and accepts a
// cell unless a cell of its 3 x 3 neighbourhood was visited before it; visiting
// stops after top_k accepted cells or at the first brightness below the
// threshold.  A cell is therefore accepted iff it precedes all of its neighbours
// in the visiting order, i.e. it is a strict local maximum of the key
//     key = (bits(|P|) << 32) | (0xFFFFFFFF - t*S - s)
// (brightness descending, then linear index ascending; non-negative floats
// order like their bit patterns), and the detected list is the top_k such keys
// with |P| >= threshold, in key order.  The neighbourhood wraps around both axes.
//
//  k_peak_tiles   one block per 32 x 64 tile: load the tile with a one-cell halo,
//                 mark strict local maxima (at most one per 2 x 2 block, so at most
//                 512 per tile), sort them and keep the best min(top_k, 512).
//  k_peak_select  one block per image: radix select (8 passes of 8 bits) of the
//                 top_k-th largest key among the tiles' keys, gather the keys at or
//                 above it, sort them and write the ft_peak records.
#include "ft_internal.cuh"

#define PK_TT 32
#define PK_TS 64
#define PK_CAND 512
#define PK_SEL_THREADS 1024

typedef unsigned long long u64;

__device__ __forceinline__ u64 peak_key(float v, unsigned lin) {
    return ((u64)__float_as_uint(v) << 32) | (u64)(0xFFFFFFFFu - lin);
}

__device__ __forceinline__ int wrap_mod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Bitonic sort, descending, of n (power of two) keys in shared memory.
__device__ void bitonic_desc(u64* v, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool desc = (i & k) == 0;
                    const u64 x = v[i], y = v[ixj];
                    if (desc ? (x < y) : (x > y)) {
                        v[i] = y;
                        v[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256)
k_peak_tiles(const float* __restrict__ map, int Hp, int S, int KT, float thr, u64* __restrict__ keys) {
    __shared__ float tile[(PK_TT + 2) * (PK_TS + 2)];
    __shared__ u64 cand[PK_CAND];
    __shared__ int ncand;
    const int img = blockIdx.z;
    const int t0 = blockIdx.y * PK_TT;
    const int s0 = blockIdx.x * PK_TS;
    const float* m = map + (size_t)img * Hp * S;

    for (int idx = threadIdx.x; idx < (PK_TT + 2) * (PK_TS + 2); idx += blockDim.x) {
        const int r = idx / (PK_TS + 2);
        const int c = idx % (PK_TS + 2);
        const int t = wrap_mod(t0 + r - 1, Hp);
        const int s = wrap_mod(s0 + c - 1, S);
        tile[idx] = fabsf(m[(size_t)t * S + s]);
    }
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();

    for (int idx = threadIdx.x; idx < PK_TT * PK_TS; idx += blockDim.x) {
        const int r = idx / PK_TS;
        const int c = idx % PK_TS;
        const int t = t0 + r;
        const int s = s0 + c;
        if (t >= Hp || s >= S) continue;
        const float v = tile[(r + 1) * (PK_TS + 2) + c + 1];
        if (!(v >= thr)) continue;
        const unsigned lin = (unsigned)t * (unsigned)S + (unsigned)s;
        const u64 key = peak_key(v, lin);
        bool is_max = true;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
#pragma unroll
            for (int dc = -1; dc <= 1; ++dc) {
                if (dr == 0 && dc == 0) continue;
                const unsigned nl = (unsigned)wrap_mod(t + dr, Hp) * (unsigned)S +
                                    (unsigned)wrap_mod(s + dc, S);
                if (nl == lin) continue;
                const float nv = tile[(r + 1 + dr) * (PK_TS + 2) + c + 1 + dc];
                if (peak_key(nv, nl) > key) is_max = false;
            }
        }
        if (is_max) {
            const int pos = atomicAdd(&ncand, 1);
            if (pos < PK_CAND) cand[pos] = key;
        }
    }
    __syncthreads();
    const int n = min(ncand, PK_CAND);
    for (int i = threadIdx.x; i < PK_CAND; i += blockDim.x)
        if (i >= n) cand[i] = 0ull;
    __syncthreads();
    bitonic_desc(cand, PK_CAND);
    u64* out = keys + ((size_t)img * gridDim.y * gridDim.x + (size_t)blockIdx.y * gridDim.x + blockIdx.x) * KT;
    for (int i = threadIdx.x; i < KT; i += blockDim.x) out[i] = cand[i];
}

__global__ void __launch_bounds__(PK_SEL_THREADS)
k_peak_select(const u64* __restrict__ keys, int n, int K, int Hp, int S, ft_peak* __restrict__ out,
              int32_t* __restrict__ count) {
    __shared__ unsigned hist[256];
    __shared__ u64 sel[FT_MAX_TOPK];
    __shared__ u64 prefix, mask;
    __shared__ int remaining, nsel, all_valid;
    const int img = blockIdx.x;
    const u64* kk = keys + (size_t)img * n;
    if (threadIdx.x == 0) {
        prefix = 0ull;
        mask = 0ull;
        remaining = K;
        all_valid = 0;
        nsel = 0;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        const u64 pf = prefix, mk = mask;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const u64 key = kk[i];
            if (key != 0ull && (key & mk) == pf) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned cum = 0;
            int d = -1;
            for (int dd = 255; dd >= 0; --dd) {
                if (cum + hist[dd] >= (unsigned)remaining) { d = dd; break; }
                cum += hist[dd];
            }
            if (d < 0) {
                all_valid = 1;                      // fewer than K valid keys
            } else {
                remaining -= (int)cum;
                prefix |= (u64)d << shift;
                mask |= 0xFFull << shift;
            }
        }
        __syncthreads();
        if (all_valid) break;
    }
    const u64 thr_key = all_valid ? 1ull : prefix;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 key = kk[i];
        if (key != 0ull && key >= thr_key) {
            const int pos = atomicAdd(&nsel, 1);
            if (pos < FT_MAX_TOPK) sel[pos] = key;
        }
    }
    __syncthreads();
    const int cnt = min(min(nsel, K), FT_MAX_TOPK);
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    for (int i = threadIdx.x; i < Kp; i += blockDim.x)
        if (i >= cnt) sel[i] = 0ull;
    __syncthreads();
    bitonic_desc(sel, Kp);
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        ft_peak p;
        if (i < cnt) {
            const u64 key = sel[i];
            const unsigned lin = 0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull);
            p.t = (int)(lin / (unsigned)S);
            p.s = (int)(lin % (unsigned)S);
            p.value = __uint_as_float((unsigned)(key >> 32));
            p.k = 2.0f * (float)(p.s - S / 2) / (float)S;
            p.b = (float)(p.t - Hp / 2);
        } else {
            p.t = 0; p.s = 0; p.value = 0.f; p.k = 0.f; p.b = 0.f;
        }
        out[(size_t)img * K + i] = p;
    }
    if (threadIdx.x == 0) count[img] = cnt;
}

static int kt_of(int top_k) { return top_k < PK_CAND ? top_k : PK_CAND; }

static dim3 tile_grid(int Hp, int S, int batch) {
    return dim3((S + PK_TS - 1) / PK_TS, (Hp + PK_TT - 1) / PK_TT, batch);
}

size_t peaks_key_bytes(int Hp, int S, int batch, int top_k) {
    const dim3 g = tile_grid(Hp, S, 1);
    return (size_t)batch * g.x * g.y * kt_of(top_k) * sizeof(u64);
}

cudaError_t launch_peak_tiles(const float* map, int Hp, int S, int batch, int top_k, float threshold,
                              unsigned long long* keys, cudaStream_t st) {
    k_peak_tiles<<<tile_grid(Hp, S, batch), 256, 0, st>>>(map, Hp, S, kt_of(top_k), threshold, keys);
    return cudaGetLastError();
}

cudaError_t launch_peak_select(const unsigned long long* keys, int Hp, int S, int batch, int top_k,
                               ft_peak* out, int32_t* count, cudaStream_t st) {
    const dim3 g = tile_grid(Hp, S, 1);
    const int n = (int)(g.x * g.y) * kt_of(top_k);
    k_peak_select<<<batch, PK_SEL_THREADS, 0, st>>>(keys, n, top_k, Hp, S, out, count);
    return cudaGetLastError();
}
