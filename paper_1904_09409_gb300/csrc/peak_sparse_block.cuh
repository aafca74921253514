// The peak pass from tile maxima (Sec. 4.4) for one map, run by one block: the
// shared pieces of k_peak_sparse.cu (one block per map of a uniform batch) and
// k_batch.cu (one block per map of a mixed-size batch).  What it computes and
// why the result equals the dense list is described in k_peak_sparse.cu.
#pragma once

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


// One map's pass, run by a whole block of nw = blockDim.x / 32 warps: m is the
// map [Hp][S], tmax its tile maxima [nty][ntx] (tiles of TH x 2^logTW cells),
// out / count its K records and its count; spsm is sparse_smem(...) bytes of
// shared memory, sh the block's shared bookkeeping.
__device__ __forceinline__ void peak_sparse_block(const float* __restrict__ m, const unsigned* __restrict__ tmax,
                                                  int Hp, int S, int TH, int logTW, int nty, int ntx, int K,
                                                  float thr, ft_peak* __restrict__ out, int32_t* __restrict__ count,
                                                  unsigned char* spsm, SparseShared& sh) {
    const int TW = 1 << logTW;
    const int cells = TH * TW;
    const int nw = blockDim.x >> 5;                    // warps = tiles per batch
    const int capc = K + nw * (cells / 4);
    const int pitch = TW + 2;                          // staged row: columns s0 - 1 .. s0 + TW
    u64* cand = reinterpret_cast<u64*>(spsm);
    u64* keep = cand + capc;
    int* list = reinterpret_cast<int*>(keep + next_pow2(K));
    const int ntiles = nty * ntx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* stg0 = reinterpret_cast<float*>(list + SP_LIST);
    float* stg = stg0 + (size_t)warp * (TH + 2) * pitch;
    const unsigned* tm = tmax;
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
                        x[u] = (cok && r < th + 2 && FT_IN(t, Hp, FT_DBG_PEAK_STAGE) && FT_IN(sc, S, FT_DBG_PEAK_STAGE))
                                   ? fabsf(__ldg(m + (size_t)t * S + sc))
                                   : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int r = rb + u * spp;
                        if (cok && r < th + 2 && FT_IN(r * pitch + c, (TH + 2) * pitch, FT_DBG_PEAK_STAGE))
                            stg[r * pitch + c] = x[u];
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
    write_peaks(keep, n, K, Hp, S, out, count, 0);
}

