// The peak pass from tile maxima (Sec. 4.4) for one map, run by one block: the
// shared pieces of k_peak_sparse.cu (one block per map of a uniform batch) and
// k_batch.cu (one block per map of a mixed-size batch).  What it computes and
// why the result equals the dense list is described in k_peak_sparse.cu.
#pragma once

#include "peaks_common.cuh"

#define SP_LIST 2048        // tiles listed at once
#define SP_CHUNK 1024       // tiles examined per listing pass (the list is run when it could overflow)

struct SparseShared {
    SelState st;            // exact radix selection (top_k > 32)
    int ncand;              // candidates in cand[]
    int nlist;              // tiles in list[]
    unsigned tbits;         // round 1 takes the valid tiles with a maximum >= this (bits)
    unsigned kth_bits;
    float bound;            // a cell below this cannot be one of the top_k peaks
    unsigned wbest[32];     // per warp of a batch: its tile's largest marked value (bits + 1; 0: none)
};

__device__ __forceinline__ void sp_cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

static __host__ __device__ int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Shared memory of a block of nw warps: one staged tile per warp,
// (rows + 2) x (cols + 8) floats (columns s0 - 4 .. s0 + cols + 3, so that
// interior tiles are copied as aligned float4 rows), cand[top_k + nw cells / 4],
// keep[next_pow2(top_k)], the warps' sorted lists mrg[nw][32], list[SP_LIST],
// then the image's tile maxima when there are at most SP_TM_SMEM tiles (they
// are read on every pass).
#define SP_TM_SMEM 8192
static size_t sparse_smem(int rows, int cols, int K, int nw, int ntiles) {
    const size_t stage = (size_t)nw * (rows + 2) * (cols + 8) * sizeof(float);
    const size_t cand = (size_t)K + (size_t)nw * rows * cols / 4;
    const size_t tms = ntiles <= SP_TM_SMEM ? (size_t)ntiles * sizeof(unsigned) : 0;
    return ((stage + 15) & ~(size_t)15) + (cand + next_pow2(K) + (size_t)nw * 32) * sizeof(u64) +
           SP_LIST * sizeof(int) + tms;
}

// One warp's descending sort of 32 values, one per lane (bitonic network over
// shuffles; blocks of k lanes alternate descending / ascending, the last merge
// is descending).
template <typename T>
__device__ __forceinline__ T warp_sort_desc(T key, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const T other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool keep_max = ((lane & j) == 0) == ((lane & k) == 0);
            key = keep_max ? (key > other ? key : other) : (key < other ? key : other);
        }
    return key;
}

// One warp: the descending top 32 of two descending lists a, b (lane i holds
// the i-th largest).  max(a[i], b[31 - i]) holds them as a bitonic sequence;
// one descending bitonic merge sorts it.
template <typename T>
__device__ __forceinline__ T warp_merge_top(T a, T b, int lane) {
    const T br = __shfl_sync(0xffffffffu, b, 31 - lane);
    T key = a > br ? a : br;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const T other = __shfl_xor_sync(0xffffffffu, key, j);
        key = (lane & j) == 0 ? (key > other ? key : other) : (key < other ? key : other);
    }
    return key;
}

// Whole block: the descending lists mrg[w][0..32) of warps w < nl (nl a power
// of two, at most the block's warps) merged pairwise in log2(nl) levels; the
// descending top 32 of all of them ends in mrg[0][0..32).
template <typename T>
__device__ void block_merge_top(T* mrg, int nl, int warp, int lane) {
    for (int span = 1; span < nl; span <<= 1) {
        __syncthreads();
        if ((warp & (2 * span - 1)) == 0 && warp + span < nl)
            mrg[warp * 32 + lane] = warp_merge_top(mrg[warp * 32 + lane], mrg[(warp + span) * 32 + lane], lane);
    }
    __syncthreads();
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
    const int P = TW + 8;                              // staged row: columns s0 - 4 .. s0 + TW + 3
    const size_t stage_bytes = ((size_t)nw * (TH + 2) * P * sizeof(float) + 15) & ~(size_t)15;
    float* stg0 = reinterpret_cast<float*>(spsm);
    u64* cand = reinterpret_cast<u64*>(spsm + stage_bytes);
    u64* keep = cand + capc;
    u64* mrg = keep + next_pow2(K);                    // [nw][32]
    int* list = reinterpret_cast<int*>(mrg + nw * 32);
    const int ntiles = nty * ntx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* stg = stg0 + (size_t)warp * (TH + 2) * P;
    const unsigned* tm = tmax;
    // interior tiles are staged as float4 rows: TW / 4 + 2 vectors per row
    const int V = (TW >> 2) + 2;
    const bool vec = (TW & 3) == 0 && V <= 32 && (S & 3) == 0 && (reinterpret_cast<size_t>(m) & 15) == 0;
    auto valid = [&](unsigned b) { return __uint_as_float(b) >= thr; };

    if (threadIdx.x == 0) {
        sh.ncand = 0;
        sh.nlist = 0;
        sh.bound = thr;
    }
    // the tile maxima, copied once when they fit (all loads in flight); then T,
    // the nw-th largest valid maximum (+1 so that 0 means none): every warp
    // sorts chunks of 32 maxima with shuffles and keeps the best 32, and a
    // merge tree over the warps leaves the best 32 of the image
    {
        unsigned* tms = reinterpret_cast<unsigned*>(list + SP_LIST);
        if (ntiles <= SP_TM_SMEM) {
            for (int i = threadIdx.x; i < ntiles; i += blockDim.x) tms[i] = tm[i];
            tm = tms;
        }
        __syncthreads();
        unsigned* m32 = reinterpret_cast<unsigned*>(mrg);
        unsigned run = 0u;
        for (int c0 = warp; c0 * 32 < ntiles; c0 += 4 * nw) {
            unsigned v[4];                             // four independent sorts in flight
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = (c0 + u * nw) * 32 + lane;
                const unsigned b = i < ntiles ? tm[i] : 0u;
                v[u] = warp_sort_desc((i < ntiles && valid(b)) ? b + 1u : 0u, lane);   // b + 1 fits: b >= 0
            }
            const unsigned a = warp_merge_top(warp_merge_top(v[0], v[1], lane), warp_merge_top(v[2], v[3], lane), lane);
            run = c0 == warp ? a : warp_merge_top(run, a, lane);
        }
        m32[warp * 32 + lane] = run;
        block_merge_top(m32, nw, warp, lane);
        const unsigned T = m32[nw - 1];
        if (threadIdx.x == 0) sh.tbits = T == 0u ? 0u : T - 1u;    // fewer than nw: every valid tile
        __syncthreads();
    }

    // test layout: lanes as rpp row groups of cw columns, cpl columns and rh
    // rows per lane; bit k rh + i of a lane's mask is row g rh + i of column
    // cl + cw k of the tile (rh cpl = cells / 32 <= 64)
    const int cw = min(TW, 32), rpp = 32 / cw, cl = lane & (cw - 1);
    const int rh = TH / rpp, g = lane / cw, cpl = TW / cw;

    // warp: the strict local maxima of tile `tile` with |P| >= bound, as the
    // lanes' masks; returns the warp's largest marked value (bits + 1, 0: none).
    // The tile and its halo (wrapped) are first copied to the warp's staging
    // area: interior tiles as aligned 16-byte rows by cp.async (columns
    // s0 - 4 .. s0 + TW + 3, all copies of a lane in flight at once), tiles at
    // the left or right edge cell by cell (columns s0 - 1 .. s0 + tw, wrapped);
    // every read of the staged cells takes |P|.
    auto test_tile = [&](int tile, float bound, unsigned long long& mask) -> unsigned {
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int t0 = ty * TH, s0 = tx * TW;
        const int th = min(TH, Hp - t0), tw = min(TW, S - s0);      // ragged last tiles
        const int nr = th + 2;
        if (vec && s0 >= 4 && s0 + TW + 4 <= S) {
            // 16-byte asynchronous copies straight into shared memory
            const int lpr = next_pow2(V), rpp = 32 / lpr;
            const int v = lane & (lpr - 1);
            const float* mb = m + (s0 - 4) + 4 * v;
            if (v < V)
                for (int r = lane / lpr; r < nr; r += rpp) {
                    int t = t0 - 1 + r;
                    t = t < 0 ? t + Hp : (t >= Hp ? t - Hp : t);
                    if (FT_IN(t, Hp, FT_DBG_PEAK_STAGE) && FT_IN(r * P + 4 * v + 3, (TH + 2) * P, FT_DBG_PEAK_STAGE))
                        sp_cp_async16(stg + r * P + 4 * v, mb + (size_t)t * S);
                }
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        } else {
            const int sw = min(32, next_pow2(tw + 2)), spp = 32 / sw;
            const int sl = lane & (sw - 1), srow = lane / sw;
            for (int c = sl; c < sw * ((tw + 1 + sw) / sw); c += sw) {
                const bool cok = c < tw + 2;
                int sc = s0 - 1 + c;
                sc = sc < 0 ? sc + S : (sc >= S ? sc - S : sc);
                for (int rb = srow; rb < nr; rb += 16 * spp) {
                    float x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int r = rb + u * spp;
                        int t = t0 - 1 + r;
                        t = t < 0 ? t + Hp : (t >= Hp ? t - Hp : t);
                        x[u] = (cok && r < nr && FT_IN(t, Hp, FT_DBG_PEAK_STAGE) && FT_IN(sc, S, FT_DBG_PEAK_STAGE))
                                   ? fabsf(__ldg(m + (size_t)t * S + sc))
                                   : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int r = rb + u * spp;
                        if (cok && r < nr && FT_IN(r * P + c + 3, (TH + 2) * P, FT_DBG_PEAK_STAGE))
                            stg[r * P + c + 3] = x[u];
                    }
                }
            }
        }
        __syncwarp();
        // a lane walks down its rows with a three-row window of columns
        // c - 1 .. c + 1, compares each cell with the maximum of its 8
        // neighbours (the exact index order only for ties with that maximum)
        // and sets one mask bit per strict local maximum
        mask = 0ull;
        unsigned best = 0u;
        for (int k = 0; k < cpl; ++k) {
            const int c = cl + cw * k;
            const float* col = stg + (c + 4) + g * rh * P;       // staged row of tile row g rh - 1
            float l0 = fabsf(col[-1]), m0 = fabsf(col[0]), r0 = fabsf(col[1]);
            float l1 = fabsf(col[P - 1]), m1 = fabsf(col[P]), r1 = fabsf(col[P + 1]);
            float h0 = fmaxf(fmaxf(l0, m0), r0);
#pragma unroll 4
            for (int i = 0; i < rh; ++i) {
                const float* p2 = col + (i + 2) * P;
                const float l2 = fabsf(p2[-1]), m2 = fabsf(p2[0]), r2 = fabsf(p2[1]);
                const float h2 = fmaxf(fmaxf(l2, m2), r2);
                const float nmax = fmaxf(fmaxf(h0, h2), fmaxf(l1, r1));
                const float v = m1;
                const int r = g * rh + i;
                bool ok = r < th && c < tw && v >= bound && v >= nmax;
                if (ok && v == nmax) {
                    // exact tie: a tied neighbour precedes iff its linear index is smaller
                    const int t = t0 + r, sc = s0 + c;
                    const unsigned lin = (unsigned)t * (unsigned)S + (unsigned)sc;
                    const float* cp = col + (i + 1) * P;
#pragma unroll
                    for (int a = -1; a <= 1; ++a)
#pragma unroll
                        for (int b = -1; b <= 1; ++b) {
                            if ((a == 0 && b == 0) || fabsf(cp[a * P + b]) != v) continue;
                            int tn = t + a, sn = sc + b;
                            tn = tn < 0 ? tn + Hp : (tn >= Hp ? tn - Hp : tn);
                            sn = sn < 0 ? sn + S : (sn >= S ? sn - S : sn);
                            const unsigned nl = (unsigned)tn * (unsigned)S + (unsigned)sn;
                            if (nl != lin && nl < lin) ok = false;
                        }
                }
                if (ok) {
                    mask |= 1ull << (k * rh + i);
                    best = max(best, __float_as_uint(v) + 1u);
                }
                h0 = fmaxf(fmaxf(l1, m1), r1);
                l1 = l2; m1 = m2; r1 = r2;
            }
        }
        return __reduce_max_sync(0xffffffffu, best);
    };

    // warp, after test_tile on the same tile: the marked cells with |P| >= cut
    // are appended to cand[] (one atomic for the warp).  The staging area is
    // reused by the warp's next tile.
    auto append_tile = [&](int tile, float cut, unsigned long long mask) {
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int t0 = ty * TH, s0 = tx * TW;
        unsigned long long keepm = 0ull;
        for (unsigned long long mk = mask; mk; mk &= mk - 1ull) {
            const int bit = __ffsll((long long)mk) - 1, k = bit / rh, i = bit - k * rh;
            if (fabsf(stg[(g * rh + i + 1) * P + cl + cw * k + 4]) >= cut) keepm |= 1ull << bit;
        }
        {
            const int cnt = __popcll(keepm);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int base = 0;
            if (lane == 31 && incl) base = atomicAdd(&sh.ncand, incl);
            base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
            for (unsigned long long mk = keepm; mk; mk &= mk - 1ull) {
                const int bit = __ffsll((long long)mk) - 1, k = bit / rh, i = bit - k * rh;
                const int c = cl + cw * k;
                const unsigned lin = (unsigned)(t0 + g * rh + i) * (unsigned)S + (unsigned)(s0 + c);
                cand[base++] = peak_key(fabsf(stg[(g * rh + i + 1) * P + c + 4]), lin);
            }
        }
        __syncwarp();
    };

    // whole block: exactly the best K candidates stay, the bound becomes value(kth)
    auto compact = [&]() {
        const int n = sh.ncand;
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
            sh.bound = fmaxf(sh.bound, __uint_as_float(sh.kth_bits));
        }
        __syncthreads();
    };

    // whole block, top_k <= 32: cand[] becomes its best min(K, ncand) keys in
    // descending order (each warp sorts chunks of 32 and keeps the best 32 of
    // its chunks, then the warps' lists are merged); with K of them the bound
    // becomes value(kth)
    auto keep_best = [&]() {
        const int n = sh.ncand;
        u64 run = 0ull;
        for (int c = warp; c * 32 < n; c += nw) {
            const int i = c * 32 + lane;
            const u64 v = warp_sort_desc(i < n ? cand[i] : 0ull, lane);
            run = c == warp ? v : warp_merge_top(run, v, lane);
        }
        const int nl = next_pow2(min(nw, (n + 31) / 32));
        if (warp < nl) mrg[warp * 32 + lane] = run;
        block_merge_top(mrg, nl, warp, lane);
        const int k = min(n, K);
        if (threadIdx.x < k) cand[threadIdx.x] = mrg[threadIdx.x];
        if (threadIdx.x == 0) {
            sh.ncand = k;
            if (k == K) sh.bound = fmaxf(sh.bound, __uint_as_float((unsigned)(mrg[K - 1] >> 32)));
        }
        __syncthreads();
    };

    // whole block: the tiles list[0..nlist), one per warp and batch, those whose
    // maximum still reaches the bound.  After each batch the candidates are cut
    // to the best K (for top_k <= 32 sorted, at every batch; else by radix
    // selection once there are K), which raises the bound and leaves room in
    // cand[] for the next batch.
    auto run_list = [&]() {
        const int nl = sh.nlist;
        for (int b0 = 0; b0 < nl; b0 += nw) {
            const float bound = sh.bound;
            const int j = b0 + warp;
            int tile = -1;
            unsigned long long mask = 0ull;
            unsigned best = 0u;
            if (j < nl && __uint_as_float(tm[list[j]]) >= bound) {
                tile = list[j];
                best = test_tile(tile, bound, mask);
            }
            // the K-th largest of the warps' best values (distinct candidates of
            // distinct tiles) is a lower bound of value(kth): only the marked
            // cells at or above it are appended
            if (lane == 0) sh.wbest[warp] = best;
            __syncthreads();
            float cut = bound;
            if (K <= nw) {
                unsigned lk;
                if (K == nw) {
                    lk = __reduce_min_sync(0xffffffffu, lane < nw ? sh.wbest[lane] : 0xFFFFFFFFu);
                } else {
                    const unsigned wb = warp_sort_desc(lane < nw ? sh.wbest[lane] : 0u, lane);
                    lk = __shfl_sync(0xffffffffu, wb, K - 1);
                }
                if (lk != 0u) cut = fmaxf(cut, __uint_as_float(lk - 1u));
            }
            if (tile >= 0) append_tile(tile, cut, mask);
            __syncthreads();
            if (K <= 32)
                keep_best();
            else if (sh.ncand >= K)
                compact();
        }
    };

    // whole block: list and run every valid tile whose maximum b satisfies
    // want(b) and reaches the bound.  Tiles are examined SP_CHUNK at a time and
    // appended to one list, which is run when another chunk could overflow it
    // and at the end (so that a short list runs as few full batches).
    auto run_tiles = [&](auto want) {
        if (threadIdx.x == 0) sh.nlist = 0;
        __syncthreads();
        for (int base = 0; base < ntiles; base += SP_CHUNK) {
            const float bound = sh.bound;
            for (int i0 = base + (threadIdx.x & ~31); i0 < min(ntiles, base + SP_CHUNK); i0 += blockDim.x) {
                const int i = i0 + lane;
                bool w = false;
                if (i < ntiles) {
                    const unsigned b = tm[i];
                    w = valid(b) && want(b) && __uint_as_float(b) >= bound;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, w);
                if (bal) {
                    int pos = 0;
                    if (lane == 0) pos = atomicAdd(&sh.nlist, __popc(bal));
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    if (w) list[pos + __popc(bal & ((1u << lane) - 1u))] = i;
                }
            }
            __syncthreads();
            if (sh.nlist > 0 && (sh.nlist > SP_LIST - SP_CHUNK || base + SP_CHUNK >= ntiles)) {
                run_list();
                __syncthreads();
                if (threadIdx.x == 0) sh.nlist = 0;
                __syncthreads();
            }
        }
    };

    // round 1: the valid tiles with a maximum >= T (at least nw of them, the nw
    // brightest among them)
    const unsigned tb = sh.tbits;
    run_tiles([&](unsigned b) { return b >= tb; });

    // round 2: every other tile that can still hold one of the top_k peaks
    // (skipped when no tile's maximum reaches the bound)
    {
        const float bound = sh.bound;
        bool any = false;
        for (int i = threadIdx.x; i < ntiles && !any; i += blockDim.x) {
            const unsigned b = tm[i];
            any = valid(b) && b < tb && __uint_as_float(b) >= bound;
        }
        if (__syncthreads_or(any)) run_tiles([&](unsigned b) { return b < tb; });
    }

    // the list: the best min(K, ncand) keys, sorted descending (for top_k <= 32
    // cand[] already is; else up to 32 keys in one warp's registers, more by a
    // block bitonic sort)
    __syncthreads();
    const int n = sh.ncand;                            // <= K
    if (K <= 32) {
        write_peaks(cand, n, K, Hp, S, out, count, 0);
        return;
    }
    if (n <= 32) {
        if (warp == 0) {
            const u64 key = warp_sort_desc(lane < n ? cand[lane] : 0ull, lane);
            if (lane < n) keep[lane] = key;            // the zero padding sorts last
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
