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
//   round 1  the brightest tiles, about one per warp of the block: every valid
//            tile (M[j] >= threshold) with M[j] >= T, where each thread takes
//            the largest valid maximum among the tiles it copies and T is the
//            nw-th largest of those (one shuffle sort per warp, then a merge
//            tree over the warps).  At least nw tiles reach T, and so does
//            every tile among the nw brightest;
//   round 2  every other valid tile with M[j] >= the bound.
// Warps take one tile each per batch, staged in shared memory with its one-cell
// halo (interior tiles as aligned float4 rows, all loads of a lane in flight at
// once; edge tiles cell by cell with the wrap).  After each batch the
// candidates are cut to the best K, and the bound becomes value(kth): for
// top_k <= 32 every warp sorts chunks of 32 keys with shuffles and keeps the
// best 32, and a merge tree over the warps leaves the best K sorted (so the
// final list needs no further sort); for larger top_k, radix selection once
// there are K candidates.  Every cell of a processed tile gets the exact test
// of k_peak_tiles (neighbours across tile borders and around the wrap), so the
// list equals the dense one: keys are distinct, and every key of the dense list
// lies in a tile that is processed and is at or above the bound when it is
// tested.
//
// Capacity: two cells of one 2 x 2 block are neighbours, so a tile of r x c cells
// holds at most r c / 4 strict local maxima; a batch (one tile per warp) adds at
// most warps x r c / 4 candidates to the top_k kept.
#include "peak_sparse_block.cuh"

__global__ void __launch_bounds__(1024)
k_peak_sparse(const float* __restrict__ map, const unsigned* __restrict__ tmax, int Hp, int S, int TH, int logTW,
              int nty, int ntx, int K, float thr, ft_peak* __restrict__ out, int32_t* __restrict__ count) {
    extern __shared__ __align__(16) unsigned char spsm[];
    __shared__ SparseShared sh;
    pdl_wait();
    pdl_trigger();                                     // step 4 is complete: the next launch may be placed
    const int img = blockIdx.x;
    peak_sparse_block(map + (size_t)img * Hp * S, tmax + (size_t)img * nty * ntx, Hp, S, TH, logTW, nty, ntx, K, thr,
                      out + (size_t)img * K, count + img, spsm, sh);
}

FT_DEBUG_READER(ft_debug_read_peak_sparse)

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
    if (rows * cols > 64 * 32) return 0;                          // a lane's cells fit one 64-bit mask
    for (int nw = 32; nw >= 8; nw /= 2)
        if (sparse_smem(rows, cols, top_k, nw, 0) + sizeof(SparseShared) + SP_TM_SMEM * sizeof(unsigned) <=
            (size_t)optin)
            return nw;
    return 0;
}

bool peak_sparse_fits(int tile_rows, int tile_cols, int top_k) { return sparse_warps(tile_rows, tile_cols, top_k) > 0; }

cudaError_t launch_peak_sparse(const float* map, const unsigned* tmax, int Hp, int S, int tile_rows, int tile_cols,
                               int batch, int top_k, float threshold, ft_peak* out, int32_t* count, cudaStream_t st,
                               bool pdl) {
    const int nw = sparse_warps(tile_rows, tile_cols, top_k);
    if (nw == 0) return cudaErrorInvalidValue;
    int logTW = 0;
    while ((1 << logTW) < tile_cols) ++logTW;
    const int nty = (Hp + tile_rows - 1) / tile_rows, ntx = (S + tile_cols - 1) / tile_cols;
    const size_t sm = sparse_smem(tile_rows, tile_cols, top_k, nw, nty * ntx);
    cudaError_t e = cudaFuncSetAttribute(k_peak_sparse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return launch_maybe_pdl(k_peak_sparse, dim3(batch), dim3(nw * 32), sm, st, pdl, map, tmax, Hp, S, tile_rows,
                            logTW, nty, ntx, top_k, threshold, out, count);
}
