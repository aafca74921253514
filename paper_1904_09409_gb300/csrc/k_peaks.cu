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
//                 512 per tile; neighbour indices are computed only to break exact
//                 ties), and keep the best min(top_k, 512) by radix selection.
//  k_peak_tiles_fast  the same for maps with S % 128 == 0 and H' % 32 == 0, one
//                 block per tile of 64 x 128 cells (32 x 128 when H' is not a
//                 multiple of 64; image index fastest in the grid): the
//                 tile and its halo are copied with cp.async, each lane tests 4
//                 columns of 4 rows against the max of their 8 neighbours (exact
//                 ties alone take the index comparison), candidates are appended
//                 per warp with one scan (at most rows x 32 per tile).  The tile's
//                 best min(top_k, rows x 32) keys go to the tile's own slots or, for large
//                 maps, are appended to the image's key list (one atomic per
//                 tile); a per-image running bound of the top_k-th value lets
//                 later tiles drop dimmer candidates early.
//  k_peak_select  one block per image: radix selection of the top_k keys among
//                 the tiles' keys (the appended list, or every tile's slots for
//                 the generic tiles), then a bitonic sort of those top_k and the
//                 ft_peak records.
//
// Radix selection (cta_select): MSB-first passes over 8-bit digits of the
// 64-bit keys; a pass histograms the digit of the keys that share the prefix
// chosen so far, a warp scan finds the digit where the top_k boundary falls, and
// the search stops as soon as that digit's bin is taken whole.  Keys are
// distinct, so the selected set has exactly min(top_k, #keys) elements.
#include "peaks_common.cuh"

#define PK_TT 32
#define PK_TS 64
#define PK_CAND 512
#define PK_TILE_THREADS 256
#define PK_SEL_THREADS 1024

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(PK_TILE_THREADS)
k_peak_tiles(const float* __restrict__ map, int Hp, int S, int KT, float thr, u64* __restrict__ keys) {
    __shared__ float tile[(PK_TT + 2) * (PK_TS + 2)];
    __shared__ u64 cand[PK_CAND];
    __shared__ int ncand;
    __shared__ SelState st;
    const int img = blockIdx.z;
    const int t0 = blockIdx.y * PK_TT;
    const int s0 = blockIdx.x * PK_TS;
    const float* m = map + (size_t)img * Hp * S;

    for (int idx = threadIdx.x; idx < (PK_TT + 2) * (PK_TS + 2); idx += blockDim.x) {
        const int r = idx / (PK_TS + 2);
        const int c = idx - r * (PK_TS + 2);
        const int t = wrap_into(t0 + r - 1, Hp);
        const int s = wrap_into(s0 + c - 1, S);
        tile[idx] = fabsf(__ldg(m + (size_t)t * S + s));
    }
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();

    for (int idx = threadIdx.x; idx < PK_TT * PK_TS; idx += blockDim.x) {
        const int r = idx / PK_TS;
        const int c = idx - r * PK_TS;
        const int t = t0 + r;
        const int s = s0 + c;
        if (t >= Hp || s >= S) continue;
        const float* cp = tile + (r + 1) * (PK_TS + 2) + c + 1;
        const float v = *cp;
        if (!(v >= thr)) continue;
        const unsigned lin = (unsigned)t * (unsigned)S + (unsigned)s;
        bool is_max = true;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
#pragma unroll
            for (int dc = -1; dc <= 1; ++dc) {
                if (dr == 0 && dc == 0) continue;
                const float nv = cp[dr * (PK_TS + 2) + dc];
                if (nv > v) {
                    is_max = false;
                } else if (nv == v) {
                    // exact tie: the neighbour precedes iff its linear index is smaller
                    const unsigned nl = (unsigned)wrap_into(t + dr, Hp) * (unsigned)S +
                                        (unsigned)wrap_into(s + dc, S);
                    if (nl != lin && nl < lin) is_max = false;
                }
            }
        }
        if (is_max) {
            const int pos = atomicAdd(&ncand, 1);
            if (pos < PK_CAND) cand[pos] = peak_key(v, lin);
        }
    }
    __syncthreads();
    const int n = min(ncand, PK_CAND);
    u64* out = keys + ((size_t)img * gridDim.y * gridDim.x + (size_t)blockIdx.y * gridDim.x + blockIdx.x) * KT;
    if (n <= KT) {
        for (int i = threadIdx.x; i < KT; i += blockDim.x) out[i] = i < n ? cand[i] : 0ull;
        return;
    }
    cta_select(cand, n, KT, st);
    if (threadIdx.x == 0) st.count = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 key = cand[i];
        if (selected(key, st)) out[atomicAdd(&st.count, 1)] = key;
    }
}

__global__ void __launch_bounds__(PK_SEL_THREADS)
k_peak_select(const u64* __restrict__ keys, const unsigned* __restrict__ bounds, int n, int K, int Hp, int S,
              ft_peak* __restrict__ out, int32_t* __restrict__ count) {
    __shared__ u64 sel[FT_MAX_TOPK];
    __shared__ SelState st;
    const u64* kk = keys + (size_t)blockIdx.x * n;
    if (bounds) n = min(n, (int)bounds[2 * blockIdx.x + 1]);   // appended key lists hold fewer keys
    cta_select(kk, n, K, st);
    if (threadIdx.x == 0) st.count = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 key = kk[i];
        if (selected(key, st)) {
            const int pos = atomicAdd(&st.count, 1);
            if (pos < FT_MAX_TOPK) sel[pos] = key;
        }
    }
    __syncthreads();
    const int cnt = min(min(st.count, K), FT_MAX_TOPK);
    int Kp = 1;
    while (Kp < cnt) Kp <<= 1;
    for (int i = threadIdx.x; i < Kp; i += blockDim.x)
        if (i >= cnt) sel[i] = 0ull;
    __syncthreads();
    bitonic_desc(sel, Kp);
    write_peaks(sel, cnt, K, Hp, S, out, count, blockIdx.x);
}

#define PF_TS 128
#define PF_PITCH (PF_TS + 8)

// Shared memory of one register tile of TT rows: the tile with its one-cell
// halo, then the candidate list (at most one strict local maximum per 2 x 2
// block: TT * PF_TS / 4), then the scalars.
template <int TT>
struct TileLayout {
    static constexpr int CAND = TT * PF_TS / 4;
    static constexpr size_t TILE_BYTES = (size_t)(TT + 2) * PF_PITCH * sizeof(float);
    static constexpr size_t BYTES = TILE_BYTES + (size_t)CAND * sizeof(u64);
};
struct TileScalars {
    int ncand;
    unsigned kth_bits;
    unsigned base;          // first slot of this tile's keys in the image's key list
    SelState st;
};

// One block of 8 warps per tile of 8 RW rows x 128 columns; warp w tests rows
// RW w .. RW w + RW - 1, lane l columns 4 l .. 4 l + 3, walking down the rows
// with a three-row window.
template <int RW>
__device__ __forceinline__ void peak_tile_fast(const float* __restrict__ m, int Hp, int S, int KT, float thr,
                                               int ty, int tx, int tile, u64* __restrict__ out,
                                               unsigned* __restrict__ tau, unsigned* __restrict__ fill,
                                               float* tl, u64* cand, TileScalars& sh) {
    constexpr int TT = 8 * RW, CAND = TileLayout<TT>::CAND;
    static_assert(4 * RW <= 32, "one mask bit per cell of a lane");
    SelState& st = sh.st;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int t0 = ty * TT + RW * warp;                    // first of this warp's rows
    const int s0 = tx * PF_TS;
    if (threadIdx.x == 0) {
        sh.ncand = 0;
        sh.kth_bits = 0xFFFFFFFFu;
    }
    // running lower bound of the image's top_k-th peak value (see launch_peak_tiles)
    float lower = thr;
    if (tau) lower = fmaxf(lower, __uint_as_float(__ldcg(tau)));

    // the tile with its one-cell halo: TT + 2 rows of PF_TS + 2 columns (interior
    // at 16-byte aligned offset 4, halo at 3 and 4 + PF_TS), copied with cp.async
    // (16 bytes interior, 4 bytes halo); |.| is applied when read
    const int tb = ty * TT;
    for (int idx = threadIdx.x; idx < (TT + 2) * (PF_TS / 4); idx += blockDim.x) {
        const int r = idx / (PF_TS / 4);
        const int j = idx - r * (PF_TS / 4);
        const int t = wrap_into(tb - 1 + r, Hp);
        cp_async16(tl + r * PF_PITCH + 4 + 4 * j, m + (size_t)t * S + s0 + 4 * j);
    }
    if (threadIdx.x < 2 * (TT + 2)) {
        const int r = threadIdx.x >> 1;
        const int side = threadIdx.x & 1;
        const int t = wrap_into(tb - 1 + r, Hp);
        const int sc = side ? (s0 + PF_TS == S ? 0 : s0 + PF_TS) : (s0 == 0 ? S - 1 : s0 - 1);
        cp_async4(tl + r * PF_PITCH + (side ? 4 + PF_TS : 3), m + (size_t)t * S + sc);
    }
    cp_async_wait_all();
    __syncthreads();

    // row k of this warp's window (k = 0 is row t0 - 1) as |.| of columns
    // s0 + 4 lane - 1 .. s0 + 4 lane + 4
    auto row6 = [&](int k, float (&x)[6]) {
        const float* rowp = tl + (RW * warp + k) * PF_PITCH + 4 + 4 * lane;
        const float4 v = *reinterpret_cast<const float4*>(rowp);
        x[0] = fabsf(rowp[-1]);
        x[1] = fabsf(v.x);
        x[2] = fabsf(v.y);
        x[3] = fabsf(v.z);
        x[4] = fabsf(v.w);
        x[5] = fabsf(rowp[4]);
    };
    unsigned mask = 0u;                                    // bit 4 (k-1) + c: cell is a candidate
    float rm[6], r0[6], rp[6];
    row6(0, rm);
    row6(1, r0);
#pragma unroll
    for (int k = 1; k <= RW; ++k) {
        row6(k + 1, rp);
        float cm[6];                                       // max of the rows above and below
#pragma unroll
        for (int j = 0; j < 6; ++j) cm[j] = fmaxf(rm[j], rp[j]);
        const int t = t0 + k - 1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = r0[c + 1];
            const float nmax = fmaxf(fmaxf(fmaxf(cm[c], cm[c + 1]), cm[c + 2]), fmaxf(r0[c], r0[c + 2]));
            bool is_max = v >= lower && v >= nmax;
            if (is_max && v == nmax) {
                // exact tie: a tied neighbour precedes iff its linear index is smaller
                const int s = s0 + 4 * lane + c;
                const unsigned lin = (unsigned)t * (unsigned)S + (unsigned)s;
                const float nb[8] = {rm[c], rm[c + 1], rm[c + 2], r0[c], r0[c + 2], rp[c], rp[c + 1], rp[c + 2]};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (nb[j] != v) continue;
                    const int dr = j < 3 ? -1 : (j < 5 ? 0 : 1);
                    const int dc = j < 3 ? j - 1 : (j == 3 ? -1 : (j == 4 ? 1 : j - 6));
                    const unsigned nl = (unsigned)wrap_into(t + dr, Hp) * (unsigned)S +
                                        (unsigned)wrap_into(s + dc, S);
                    if (nl != lin && nl < lin) is_max = false;
                }
            }
            if (is_max) mask |= 1u << (4 * (k - 1) + c);
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            rm[j] = r0[j];
            r0[j] = rp[j];
        }
    }
    // one append per warp (only warps with candidates): exclusive scan of the lanes' counts
    const int cnt = __popc(mask);
    if (__any_sync(0xffffffffu, cnt != 0)) {
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int basepos = 0;
        if (lane == 31) basepos = atomicAdd(&sh.ncand, incl);
        basepos = __shfl_sync(0xffffffffu, basepos, 31) + incl - cnt;
        for (unsigned mk = mask; mk; mk &= mk - 1u) {      // the set bits only
            const int b = __ffs(mk) - 1;
            const int k = b >> 2, c = b & 3;
            const float v = fabsf(tl[(RW * warp + k + 1) * PF_PITCH + 4 + 4 * lane + c]);
            const unsigned lin = (unsigned)(t0 + k) * (unsigned)S + (unsigned)(s0 + 4 * lane + c);
            if (basepos < CAND) cand[basepos] = peak_key(v, lin);
            ++basepos;
        }
    }
    __syncthreads();
    const int n = min(sh.ncand, CAND);
    if (fill) {
        // the tile's min(n, KT) keys are appended to the image's key list
        if (n == 0) return;
        if (threadIdx.x == 0) sh.base = atomicAdd(fill, (unsigned)min(n, KT));
        __syncthreads();
        out += sh.base;
    } else {
        // the tile's KT slots, unused ones zero
        out += (size_t)tile * KT;
        for (int i = n + threadIdx.x; i < KT; i += blockDim.x) out[i] = 0ull;
    }
    if (n < KT) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = cand[i];
        return;
    }
    if (n == KT) {
        for (int i = threadIdx.x; i < KT; i += blockDim.x) {
            out[i] = cand[i];
            atomicMin(&sh.kth_bits, (unsigned)(cand[i] >> 32));
        }
    } else {
        cta_select(cand, n, KT, st);
        if (threadIdx.x == 0) st.count = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const u64 key = cand[i];
            if (selected(key, st)) {
                out[atomicAdd(&st.count, 1)] = key;
                atomicMin(&sh.kth_bits, (unsigned)(key >> 32));
            }
        }
    }
    // this tile alone has top_k candidates >= kth: the image's top_k-th peak is
    // at least that bright, so later tiles may drop anything dimmer
    __syncthreads();
    if (tau && threadIdx.x == 0) atomicMax(tau, sh.kth_bits);
}

// One block per tile; the image index runs fastest in the grid, so the blocks of
// the first wave cover the first tiles of every image and the later waves find
// each image's running bound already raised.
template <int RW>
__global__ void __launch_bounds__(PK_TILE_THREADS)
k_peak_tiles_fast(const float* __restrict__ map, int Hp, int S, int KT, float thr, u64* __restrict__ keys,
                  unsigned* __restrict__ bounds, int use_tau, int compact) {
    constexpr int TT = 8 * RW;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ TileScalars sh;
    const int img = blockIdx.x;
    const int tile = blockIdx.y;
    const int ntx = S / PF_TS, ntiles = ntx * (Hp / TT);
    const int ty = tile / ntx, tx = tile - ty * ntx;
    peak_tile_fast<RW>(map + (size_t)img * Hp * S, Hp, S, KT, thr, ty, tx, tile, keys + (size_t)img * ntiles * KT,
                       use_tau ? bounds + 2 * img : nullptr, compact ? bounds + 2 * img + 1 : nullptr,
                       reinterpret_cast<float*>(psm),
                       reinterpret_cast<u64*>(psm + TileLayout<TT>::TILE_BYTES), sh);
}

// register tiles: 64 rows where n_intercept allows, else 32
static bool fast_tiles(int Hp, int S) { return S % PF_TS == 0 && Hp % 32 == 0; }
static int fast_rows(int Hp) { return Hp % 64 == 0 ? 64 : 32; }

// keys kept per tile: every candidate a tile can hold when top_k exceeds it
// (a 32 x 64 tile has at most 512 strict local maxima, a register tile of 32 or
// 64 x 128 cells 1024 or 2048, both at least FT_MAX_TOPK)
static int kt_of(int Hp, int S, int top_k) {
    const int cap = fast_tiles(Hp, S) ? fast_rows(Hp) * PF_TS / 4 : PK_CAND;
    return top_k < cap ? top_k : cap;
}

// Key layout of the register tiles: every tile's KT slots (zero when unused)
// while the selection can afford to scan them all, else one appended list per
// image (one global atomic per tile, the selection reads only real keys).
#define PK_COMPACT_MIN 32768
static bool compact_keys(int Hp, int S, int top_k) {
    return (long long)(S / PF_TS) * (Hp / fast_rows(Hp)) * kt_of(Hp, S, top_k) > PK_COMPACT_MIN;
}

static dim3 tile_grid(int Hp, int S, int batch) {
    if (fast_tiles(Hp, S)) return dim3(S / PF_TS, Hp / fast_rows(Hp), batch);
    return dim3((S + PK_TS - 1) / PK_TS, (Hp + PK_TT - 1) / PK_TT, batch);
}

size_t peaks_tile_keys(int Hp, int S, int top_k) {
    const dim3 g = tile_grid(Hp, S, 1);
    return (size_t)g.x * g.y * kt_of(Hp, S, top_k);
}

static size_t key_bytes(int Hp, int S, int batch, int top_k) {
    return ((size_t)batch * peaks_tile_keys(Hp, S, top_k) * sizeof(u64) + 255) & ~(size_t)255;
}

// scratch: the tiles' keys, then per image {running bound, key count}
size_t peaks_key_bytes(int Hp, int S, int batch, int top_k) {
    return key_bytes(Hp, S, batch, top_k) + (size_t)2 * batch * sizeof(unsigned);
}

unsigned* peaks_bounds(unsigned long long* keys, int Hp, int S, int batch, int top_k) {
    return reinterpret_cast<unsigned*>(reinterpret_cast<char*>(keys) + key_bytes(Hp, S, batch, top_k));
}

// The register-only tile kernel keeps, per image, a running lower bound of the
// top_k-th peak value (as float bits): a tile that finds top_k candidates raises
// it to its own top_k-th value, and later tiles drop dimmer candidates before
// selecting.  Every such tile keeps top_k keys (top_k <= 1024 = its capacity),
// so the bound always applies.  The bounds are cleared on the stream before the
// tiles run.
cudaError_t launch_peak_tiles(const float* map, int Hp, int S, int batch, int top_k, float threshold,
                              unsigned long long* keys, unsigned* bounds, cudaStream_t st) {
    const int KT = kt_of(Hp, S, top_k);
    if (fast_tiles(Hp, S)) {
        cudaError_t e = cudaMemsetAsync(bounds, 0, (size_t)2 * batch * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        const int TT = fast_rows(Hp);
        const dim3 grid(batch, (S / PF_TS) * (Hp / TT));
        const int use_tau = KT == top_k ? 1 : 0, compact = compact_keys(Hp, S, top_k) ? 1 : 0;
        if (TT == 64) {
            const size_t sm = TileLayout<64>::BYTES;
            e = cudaFuncSetAttribute(k_peak_tiles_fast<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_peak_tiles_fast<8><<<grid, PK_TILE_THREADS, sm, st>>>(map, Hp, S, KT, threshold, keys, bounds, use_tau,
                                                                    compact);
        } else {
            k_peak_tiles_fast<4><<<grid, PK_TILE_THREADS, TileLayout<32>::BYTES, st>>>(map, Hp, S, KT, threshold, keys,
                                                                                    bounds, use_tau, compact);
        }
    }
    else {
        k_peak_tiles<<<tile_grid(Hp, S, batch), PK_TILE_THREADS, 0, st>>>(map, Hp, S, KT, threshold, keys);
    }
    return cudaGetLastError();
}

cudaError_t launch_peak_select(const unsigned long long* keys, const unsigned* bounds, int Hp, int S, int batch,
                               int top_k, ft_peak* out, int32_t* count, cudaStream_t st) {
    const bool appended = fast_tiles(Hp, S) && compact_keys(Hp, S, top_k);
    k_peak_select<<<batch, PK_SEL_THREADS, 0, st>>>(keys, appended ? bounds : nullptr,
                                                    (int)peaks_tile_keys(Hp, S, top_k), top_k, Hp, S, out, count);
    return cudaGetLastError();
}
