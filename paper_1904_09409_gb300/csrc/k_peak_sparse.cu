// Peak detection of Sec. 4.4 driven by tile maxima of |P|: the same detected
// list as launch_peak_tiles + launch_peak_select, found by reading only the
// tiles that can hold one of the top_k peaks.  The maxima come from step 4
// (launch_col_c2r_fast with a tmax buffer, ft_detect) or from k_tile_max, one
// streaming read of a given map (ft_peaks).
//
// The detected list is the top_k strict local maxima of the key
//     key = (bits(|P|) << 32) | (0xFFFFFFFF - t*S - s)
// with |P| >= threshold (the 3 x 3 neighbourhood wraps around both axes; see
// k_peaks.cu).  A peak inside tile j has |P| <= M[j], the tile's maximum.  So
// once K = top_k peaks with keys >= kth are known, a tile with M[j] < value(kth)
// cannot contribute and is never read.  One block per image:
//   round 1  the tiles with the largest maxima, one per warp of the block
//            (radix selection over the tile keys (M[j], j)), among the tiles
//            with M[j] >= threshold;
//   round 2  every other tile with M[j] >= max(threshold, value(kth)), where kth
//            is the top_k-th key found so far (all tiles with M[j] >= threshold
//            while fewer than top_k peaks are known);
// then the top_k keys sorted descending become the ft_peak records.  Warps take
// one tile each per batch, staged in shared memory with its one-cell halo;
// after a batch the candidates are cut back to the best top_k, which raises
// value(kth) for the next batch.  Every cell of a processed tile gets the exact
// test of k_peak_tiles (neighbours across tile borders and around the wrap),
// so the list equals the dense one: keys are distinct, and every key of the
// dense list lies in a tile that is processed.
//
// Capacity: two cells of one 2 x 2 block are neighbours, so a tile of r x c cells
// holds at most r c / 4 strict local maxima; a batch (one tile per warp) adds at
// most warps x r c / 4 candidates to the top_k kept.
#include "peaks_common.cuh"

#define SP_LIST 1024        // tiles listed at once (round 1: at most one per warp)

struct SparseShared {
    SelState tiles;         // round-1 selection of tiles
    SelState st;            // selection of candidates
    int ncand;              // candidates in cand[]
    int nlist;              // tiles in list[]
    int have_k;             // cand[] holds top_k keys: bound includes value(kth)
    unsigned kth_bits;
    float bound;            // a cell below this cannot be one of the top_k peaks
};

static __host__ __device__ int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Shared memory of a block of nw warps: cand[top_k + nw cells / 4],
// keep[next_pow2(top_k)], list[SP_LIST], one staged tile with its one-cell halo
// per warp, (rows + 2) x (cols + 2) floats, then the image's tile maxima when
// there are at most SP_TM_SMEM tiles (they are read on every selection pass).
#define SP_TM_SMEM 8192
static size_t sparse_smem(int rows, int cols, int K, int nw, int ntiles) {
    const size_t cand = (size_t)K + (size_t)nw * rows * cols / 4;
    const size_t stage = (size_t)nw * (rows + 2) * (cols + 2) * sizeof(float);
    const size_t tms = ntiles <= SP_TM_SMEM ? (size_t)ntiles * sizeof(unsigned) : 0;
    return (cand + next_pow2(K)) * sizeof(u64) + SP_LIST * sizeof(int) + stage + tms;
}


__global__ void __launch_bounds__(1024)
k_peak_sparse(const float* __restrict__ map, const unsigned* __restrict__ tmax, int Hp, int S, int TH, int logTW,
              int nty, int ntx, int K, float thr, ft_peak* __restrict__ out, int32_t* __restrict__ count) {
    extern __shared__ __align__(16) unsigned char spsm[];
    __shared__ SparseShared sh;
    const int TW = 1 << logTW;
    const int cells = TH * TW;
    const int nw = blockDim.x >> 5;                    // warps = tiles per batch
    const int capc = K + nw * (cells / 4);
    const int pitch = TW + 2;                          // staged row: columns s0 - 1 .. s0 + TW
    u64* cand = reinterpret_cast<u64*>(spsm);
    u64* keep = cand + capc;
    int* list = reinterpret_cast<int*>(keep + next_pow2(K));
    const int img = blockIdx.x;
    const float* m = map + (size_t)img * Hp * S;
    const int ntiles = nty * ntx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* stg0 = reinterpret_cast<float*>(list + SP_LIST);
    float* stg = stg0 + (size_t)warp * (TH + 2) * pitch;
    const unsigned* tm = tmax + (size_t)img * nty * ntx;
    if (ntiles <= SP_TM_SMEM) {                        // the tile maxima, copied once
        unsigned* tms = reinterpret_cast<unsigned*>(stg0 + (size_t)nw * (TH + 2) * pitch);
        for (int i = threadIdx.x; i < ntiles; i += blockDim.x) tms[i] = tm[i];
        tm = tms;                                      // visible after the first selection barrier
    }
    // test layout: rpp row groups of cw lanes, one column each (TW / cw columns per lane)
    const int cw = min(TW, 32), rpp = 32 / cw, cl = lane & (cw - 1);

    // round-1 key of tile i: (M, i) for tiles that reach the threshold, else 0
    auto tkey = [&](int i) -> u64 {
        const unsigned b = tm[i];
        return __uint_as_float(b) >= thr ? ((u64)b << 32) | (u64)(0xFFFFFFFFu - (unsigned)i) : 0ull;
    };

    // warp: every strict local maximum of tile `tile` with |P| >= bound is
    // appended to cand[].  The tile and its halo (wrapped) are first copied, as
    // |P|, to the warp's staging area: lanes as spp rows of sw columns (sw = the
    // staged width rounded up to a power of two, at most 32), 16 coalesced loads
    // in flight per lane.
    auto scan_tile = [&](int tile, float bound) {
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int t0 = ty * TH, s0 = tx * TW;
        const int th = min(TH, Hp - t0), tw = min(TW, S - s0);      // ragged last tiles
        {
            const int sw = min(32, next_pow2(tw + 2)), spp = 32 / sw;
            const int sl = lane & (sw - 1), srow = lane / sw;
            for (int c = sl; c < sw * ((tw + 1 + sw) / sw); c += sw) {
                const bool cok = c < tw + 2;
                int sc = s0 - 1 + c;
                sc = sc < 0 ? sc + S : (sc >= S ? sc - S : sc);
                for (int rb = srow; rb < th + 2; rb += 16 * spp) {
                    float x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int r = rb + u * spp;
                        int t = t0 - 1 + r;
                        t = t < 0 ? t + Hp : (t >= Hp ? t - Hp : t);
                        x[u] = (cok && r < th + 2) ? fabsf(__ldg(m + (size_t)t * S + sc)) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int r = rb + u * spp;
                        if (cok && r < th + 2) stg[r * pitch + c] = x[u];
                    }
                }
            }
        }
        __syncwarp();
        // Test: lanes as rpp row groups of cw columns (cpl columns each); a lane
        // walks down its rows with a three-row window of columns c - 1 .. c + 1,
        // compares each cell with the maximum of its 8 neighbours (the exact
        // index order only for ties with that maximum) and sets one mask bit per
        // strict local maximum; the warp then appends all of them with one scan.
        const int rh = TH / rpp, g = lane / cw, cpl = TW / cw;
        for (int k = 0; k < cpl; ++k) {
            const int c = cl + cw * k;
            const float* col = stg + (c + 1) + g * rh * pitch;   // staged row of tile row g rh - 1
            float l0 = col[-1], m0 = col[0], r0 = col[1];
            float l1 = col[pitch - 1], m1 = col[pitch], r1 = col[pitch + 1];
            float h0 = fmaxf(fmaxf(l0, m0), r0);
            unsigned long long mask = 0ull;
#pragma unroll 4
            for (int i = 0; i < rh; ++i) {
                const float* p2 = col + (i + 2) * pitch;
                const float l2 = p2[-1], m2 = p2[0], r2 = p2[1];
                const float h2 = fmaxf(fmaxf(l2, m2), r2);
                const float nmax = fmaxf(fmaxf(h0, h2), fmaxf(l1, r1));
                const float v = m1;
                const int r = g * rh + i;
                bool ok = r < th && c < tw && v >= bound && v >= nmax;
                if (ok && v == nmax) {
                    // exact tie: a tied neighbour precedes iff its linear index is smaller
                    const int t = t0 + r, sc = s0 + c;
                    const unsigned lin = (unsigned)t * (unsigned)S + (unsigned)sc;
                    const float* cp = col + (i + 1) * pitch;
#pragma unroll
                    for (int a = -1; a <= 1; ++a)
#pragma unroll
                        for (int b = -1; b <= 1; ++b) {
                            if ((a == 0 && b == 0) || cp[a * pitch + b] != v) continue;
                            int tn = t + a, sn = sc + b;
                            tn = tn < 0 ? tn + Hp : (tn >= Hp ? tn - Hp : tn);
                            sn = sn < 0 ? sn + S : (sn >= S ? sn - S : sn);
                            const unsigned nl = (unsigned)tn * (unsigned)S + (unsigned)sn;
                            if (nl != lin && nl < lin) ok = false;
                        }
                }
                if (ok) mask |= 1ull << i;
                h0 = fmaxf(fmaxf(l1, m1), r1);
                l1 = l2; m1 = m2; r1 = r2;
            }
            // one append for the warp: exclusive scan of the lanes' counts
            const int cnt = __popcll(mask);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int base = 0;
            if (lane == 31 && incl) base = atomicAdd(&sh.ncand, incl);
            base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
            for (unsigned long long mk = mask; mk; mk &= mk - 1ull) {
                const int i = __ffsll((long long)mk) - 1;
                const unsigned lin = (unsigned)(t0 + g * rh + i) * (unsigned)S + (unsigned)(s0 + c);
                cand[base++] = peak_key(col[(i + 1) * pitch], lin);
            }
        }
        __syncwarp();                                  // the staging area is reused by the next tile
    };

    // whole block: keep the best K candidates, raise the bound to value(kth)
    auto compact = [&]() {
        const int n = sh.ncand;
        if (n < K || (n == K && sh.have_k)) return;
        cta_select(cand, n, K, sh.st);
        if (threadIdx.x == 0) {
            sh.st.count = 0;
            sh.kth_bits = 0xFFFFFFFFu;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const u64 key = cand[i];
            if (selected(key, sh.st)) {
                keep[atomicAdd(&sh.st.count, 1)] = key;
                atomicMin(&sh.kth_bits, (unsigned)(key >> 32));
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += blockDim.x) cand[i] = keep[i];
        if (threadIdx.x == 0) {
            sh.ncand = K;
            sh.have_k = 1;
            sh.bound = fmaxf(thr, __uint_as_float(sh.kth_bits));
        }
        __syncthreads();
    };

    // whole block: the tiles list[0..nlist), one per warp and batch, those whose
    // maximum still reaches the bound
    auto run_list = [&]() {
        const int nl = sh.nlist;
        for (int b0 = 0; b0 < nl; b0 += nw) {
            const float bound = sh.bound;
            const int j = b0 + warp;
            if (j < nl) {
                const int tile = list[j];
                if (__uint_as_float(tm[tile]) >= bound) scan_tile(tile, bound);
            }
            __syncthreads();
            compact();
        }
    };

    if (threadIdx.x == 0) {
        sh.ncand = 0;
        sh.nlist = 0;
        sh.have_k = 0;
        sh.bound = thr;
    }
    // round 1: the brightest tiles, one per warp
    cta_select_by(ntiles, min(ntiles, nw), sh.tiles, tkey);
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x)
        if (selected(tkey(i), sh.tiles)) list[atomicAdd(&sh.nlist, 1)] = i;
    __syncthreads();
    run_list();

    // round 2: every other tile that can still hold one of the top_k peaks (the
    // whole round is skipped when no tile's maximum reaches the bound)
    bool any = false;
    for (int i = threadIdx.x; i < ntiles && !any; i += blockDim.x) {
        const u64 k = tkey(i);
        any = k != 0ull && !selected(k, sh.tiles) && __uint_as_float(tm[i]) >= sh.bound;
    }
    for (int base = 0; __syncthreads_or(any) && base < ntiles; base += SP_LIST) {
        __syncthreads();
        if (threadIdx.x == 0) sh.nlist = 0;
        __syncthreads();
        for (int i0 = base + (threadIdx.x & ~31); i0 < min(ntiles, base + SP_LIST); i0 += blockDim.x) {
            const int i = i0 + lane;
            bool want = false;
            if (i < ntiles) {
                const u64 k = tkey(i);
                want = k != 0ull && !selected(k, sh.tiles) && __uint_as_float(tm[i]) >= sh.bound;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, want);
            if (bal) {
                int pos = 0;
                if (lane == 0) pos = atomicAdd(&sh.nlist, __popc(bal));
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if (want) list[pos + __popc(bal & ((1u << lane) - 1u))] = i;
            }
        }
        __syncthreads();
        if (sh.nlist) run_list();
    }

    // the list: the best min(K, ncand) keys, sorted descending (up to 32 keys in
    // one warp's registers, more in shared memory)
    __syncthreads();
    const int n = sh.ncand;                            // <= K after the last compaction
    if (n <= 32) {
        if (warp == 0) {
            u64 key = lane < n ? cand[lane] : 0ull;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const u64 other = __shfl_xor_sync(0xffffffffu, key, j);
                    // blocks of k lanes alternate descending / ascending; the
                    // last merge (k = 32) is descending
                    const bool keep_max = ((lane & j) == 0) == ((lane & k) == 0);
                    key = keep_max ? (key > other ? key : other) : (key < other ? key : other);
                }
            if (lane < n) keep[lane] = key;          // the zero padding sorts last
        }
        __syncthreads();
    } else {
        const int Kp = next_pow2(n);
        for (int i = threadIdx.x; i < Kp; i += blockDim.x) keep[i] = i < n ? cand[i] : 0ull;
        __syncthreads();
        bitonic_desc(keep, Kp);
    }
    write_peaks(keep, n, K, Hp, S, out, count, img);
}

// Tile maxima of given maps: one warp per tile of PT_ROWS x PT_COLS cells (the
// last row / column of tiles ragged), lane l reading columns 2 (l mod 8) + 0, 1
// of rows l / 8 + 4 j (8-byte loads, 64 bytes per row, all 4 in flight); NaN
// counts as 0.  tmax[b][ceil(Hp / PT_ROWS)][ceil(S / PT_COLS)].
#define PT_ROWS 16
#define PT_COLS 16
__global__ void __launch_bounds__(256)
k_tile_max(const float* __restrict__ map, int Hp, int S, int nty, int ntx, unsigned* __restrict__ tmax) {
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (tile >= nty * ntx) return;
    const int lane = threadIdx.x & 31;
    const int ty = tile / ntx, tx = tile - ty * ntx;
    const int s = tx * PT_COLS + 2 * (lane & 7);
    const int t0 = ty * PT_ROWS + (lane >> 3);
    const float* m = map + (size_t)blockIdx.y * Hp * S + s;
    float2 v[PT_ROWS / 4];
#pragma unroll
    for (int j = 0; j < PT_ROWS / 4; ++j) {            // S is even, so s < S means s + 1 < S
        const int t = t0 + 4 * j;
        v[j] = (s < S && t < Hp) ? __ldg(reinterpret_cast<const float2*>(m + (size_t)t * S)) : make_float2(0.f, 0.f);
    }
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < PT_ROWS / 4; ++j) mx = fmaxf(mx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
    const unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
    if (lane == 0) tmax[((size_t)blockIdx.y * nty + ty) * ntx + tx] = u;
}

void tile_max_shape(int* tile_rows, int* tile_cols) {
    *tile_rows = PT_ROWS;
    *tile_cols = PT_COLS;
}

cudaError_t launch_tile_max(const float* map, int Hp, int S, int batch, unsigned* tmax, cudaStream_t st) {
    const int nty = (Hp + PT_ROWS - 1) / PT_ROWS, ntx = (S + PT_COLS - 1) / PT_COLS;
    const dim3 grid((nty * ntx + 7) / 8, batch);
    k_tile_max<<<grid, 256, 0, st>>>(map, Hp, S, nty, ntx, tmax);
    return cudaGetLastError();
}

// warps of the peak pass's block: 32, 16 or 8, the most whose shared memory
// fits the current device (0: none does)
static int sparse_warps(int rows, int cols, int top_k) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if ((rows * cols) % 32 != 0 || (cols & (cols - 1)) != 0) return 0;
    if (rows * (cols < 32 ? cols : 32) > 64 * 32) return 0;      // a lane's rows fit one 64-bit mask
    for (int nw = 32; nw >= 8; nw /= 2)
        if (sparse_smem(rows, cols, top_k, nw, 0) + sizeof(SparseShared) + SP_TM_SMEM * sizeof(unsigned) <=
            (size_t)optin)
            return nw;
    return 0;
}

bool peak_sparse_fits(int tile_rows, int tile_cols, int top_k) { return sparse_warps(tile_rows, tile_cols, top_k) > 0; }

cudaError_t launch_peak_sparse(const float* map, const unsigned* tmax, int Hp, int S, int tile_rows, int tile_cols,
                               int batch, int top_k, float threshold, ft_peak* out, int32_t* count, cudaStream_t st) {
    const int nw = sparse_warps(tile_rows, tile_cols, top_k);
    if (nw == 0) return cudaErrorInvalidValue;
    int logTW = 0;
    while ((1 << logTW) < tile_cols) ++logTW;
    const int nty = (Hp + tile_rows - 1) / tile_rows, ntx = (S + tile_cols - 1) / tile_cols;
    const size_t sm = sparse_smem(tile_rows, tile_cols, top_k, nw, nty * ntx);
    cudaError_t e = cudaFuncSetAttribute(k_peak_sparse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_peak_sparse<<<batch, nw * 32, sm, st>>>(map, tmax, Hp, S, tile_rows, logTW, nty, ntx, top_k, threshold, out,
                                              count);
    return cudaGetLastError();
}
