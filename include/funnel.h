/*
 * funnel.h — C ABI of the GB300 (sm_103a) funnel-transform library, libfunnel.so.
 *
 * The funnel transform (Wei, Feng & Zheng, "Funnel Transform for Straight Line
 * Detection", Sec. 3.1) maps a real grayscale image to a real slope-intercept
 * parameter map whose local maxima are the image's straight lines:
 *   step 1  1D Fourier transform along y of the zero-expanded image (eq. 16, Sec. 4.2)
 *   step 2  nonlinear variable-metric transform (NVMT) x' = (w2 / w_max) x, a 1D
 *           interpolated resampling of every kept frequency row (eqs. 17-18)
 *   step 3  1D Fourier transform along x'
 *   step 4  inverse 1D Fourier transform along w2 (eq. 19)
 * followed by |.| and the list-based peak detection of Sec. 4.4.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Sizes: image H x W; n_intercept = H' >= H (the expanded height, Sec. 4.2:
 *    (H'-H)/2 zero rows above, the rest below); n_slope = S >= W (zero insertion
 *    along x', Sec. 4.3).  W, H', S must be even; H' and S must be of the form
 *    2^a 3^b and at most FT_MAX_LENGTH.  Otherwise FT_ERR_UNSUPPORTED_SIZE.
 *  - Layouts (all row-major, densely packed, FP32):
 *      image  [batch][H][W]            row = image row, col = image column
 *      map    [batch][H'][S]           map[t][s]: intercept n = t - H'/2,
 *                                      slope index m = s - S/2, so k = 2m/S, b = n
 *                                      (eqs. 22-23, centred coordinates of the
 *                                      expanded image: x = col - W/2,
 *                                      y = row + (H'-H)/2 - H'/2)
 *  - Ownership: the caller owns every buffer it passes.  Pointers named d_* are
 *    device pointers on the plan's device; h_* are host pointers (pinned memory
 *    gives the fastest copies).  The plan owns its tables and its workspace, which
 *    grows on demand with the batch (grow = synchronise the device, free, allocate).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device calls are asynchronous and stream-ordered.  One plan may be
 *    used by one stream at a time; calls that overlap on the GPU with the same plan
 *    race on its workspace.
 *  - Errors: argument errors return synchronously without touching the GPU.  A
 *    CUDA error seen at a call returns FT_ERR_CUDA; ft_last_error() then gives
 *    the CUDA error text.  No C++ exception crosses the ABI.
 */
#ifndef FUNNEL_H
#define FUNNEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FT_MAX_LENGTH 8192   /* largest supported H' and S */
#define FT_MAX_TOPK 1024     /* largest top_k of ft_peaks */

typedef struct ft_plan_s* ft_plan;

typedef enum {
    FT_OK = 0,
    FT_ERR_INVALID_ARG = 1,      /* null pointer, batch < 0, top_k out of range, bad enum */
    FT_ERR_UNSUPPORTED_SIZE = 2, /* odd / non 2^a 3^b / too large / n_slope < W ... */
    FT_ERR_OOM = 3,              /* a device or host allocation failed */
    FT_ERR_CUDA = 4,             /* a CUDA runtime call or launch failed */
    FT_ERR_TIMEOUT = 5           /* a bounded device-side wait gave up (ft_plan_tc_errors) */
} ft_status;

/* Step 2 interpolator.  Sec. IV adopts a chirp-z (band-limited) interpolator,
 * Sec. V a linear one.  LINEAR: rows are zero outside the image columns, the
 * sample x' H' / (2 l) is split exactly into its integer floor and remainder and
 * the fraction is remainder * (1 / (2 l)) in FP32.  CUBIC: Keys' kernel,
 * a = -0.5.  FOURIER: the trigonometric interpolant of the row (Nyquist term as
 * a cosine) evaluated at the samples by a chirp-z (Bluestein) convolution of
 * length M = the smallest 2^a 3^b >= W + S, zero outside p in [-W/2, W/2-1];
 * W must then be 2^a 3^b and M <= FT_MAX_LENGTH; ft_backward runs its exact
 * transpose (the chirp-z stages conjugated in reverse order). */
typedef enum {
    FT_INTERP_LINEAR = 0,
    FT_INTERP_CUBIC = 1,
    FT_INTERP_FOURIER = 2
} ft_interp;

/* One detected peak (Sec. 4.4) with its line (eqs. 22-23):
 * t, s = map row / column; value = |P[t][s]|; k = 2 (s - S/2) / S;
 * b = t - H'/2 (intercept in centred coordinates of the expanded image). */
typedef struct {
    int32_t t;
    int32_t s;
    float value;
    float k;
    float b;
} ft_peak;

/* Create a plan for H x W images, n_slope x n_intercept maps, interpolator
 * `interp` (an ft_interp).  Builds the FP64-derived twiddle tables on the host and
 * copies them to the current CUDA device, which becomes the plan's device.
 * *out is set to NULL on failure. */
ft_status ft_plan_create(ft_plan* out, int H, int W, int n_slope, int n_intercept, int interp);

/* Parameter space of a plan (Sec. 4.1-4.3).  REGULAR: the funnel transform of
 * Sec. 3.1 (slopes in (-1, 1], eqs. 22-23).  INVERSE: its dual form (Fourier
 * transform along x, NVMT y' = (w1 / w_max) y, transform along y', inverse
 * along w1), for slopes outside (-1, 1] (eqs. 24-25).  The inverse space is
 * the regular transform of the transposed image: the map [n_intercept][n_slope]
 * then has t = b_x + n_intercept/2 (x-intercept, centred) and
 * s = n + n_slope/2 with 1/k = 2 n / n_slope; n_slope >= H and n_intercept >= W,
 * H even; ft_peak.k holds 1/k and ft_peak.b holds b_x. */
typedef enum {
    FT_SPACE_REGULAR = 0,
    FT_SPACE_INVERSE = 1
} ft_space;

/* ft_plan_create with an explicit space (ft_plan_create is the REGULAR case). */
ft_status ft_plan_create_space(ft_plan* out, int H, int W, int n_slope, int n_intercept, int interp,
                               int space);

/* Release the plan's tables and workspace (synchronises the plan's device).
 * NULL is accepted. */
ft_status ft_plan_destroy(ft_plan plan);

/* Sec. 3.1 steps 1-4: d_map[b] = P(d_img[b]) for b < batch.  batch = 0 is a
 * no-op.  d_img: [batch][H][W], d_map: [batch][H'][S], both FP32, 8-byte
 * aligned.  Launches 3 kernels on `stream`. */
ft_status ft_forward(ft_plan plan, const float* d_img, float* d_map, int batch, void* stream);

/* Exact adjoint (transpose) of ft_forward, which is linear in the image:
 * d_grad_img = A^T d_grad_map, so <A x, y> = <x, A^T y>.  Same layouts and rules
 * as ft_forward with the roles of the two buffers exchanged. */
ft_status ft_backward(ft_plan plan, const float* d_grad_map, float* d_grad_img, int batch,
                      void* stream);

/* Sec. 4.4 on |d_map| per image: the cells that no earlier-visited 3 x 3
 * neighbour precedes (order: |P| descending, then linear index t*S + s
 * ascending; the neighbourhood wraps around both axes), with |P| >= threshold,
 * the first top_k of them in that order.  d_out: [batch][top_k] ft_peak;
 * d_count: [batch] int32, the number of peaks written (< top_k when fewer pass
 * the threshold; unused slots are zeroed).  1 <= top_k <= FT_MAX_TOPK; a NaN
 * threshold is FT_ERR_INVALID_ARG.  Two launches, one of two passes with the
 * same result, whichever a cost model measured on GB300 expects to be faster
 * for this batch, map size and top_k (FT_PEAKS=sparse or dense in the
 * environment at plan creation fixes it): either the maximum of |P| per 16 x 16
 * tile (one read of the maps), then one block per map that tests only the
 * tiles whose maximum can reach the top_k (a peak never exceeds its tile's
 * maximum), brightest tiles first; or every tile's strict local maxima over
 * the whole GPU, then a per-map selection. */
ft_status ft_peaks(ft_plan plan, const float* d_map, int batch, int top_k, float threshold,
                   ft_peak* d_out, int32_t* d_count, void* stream);

/* Detection on device buffers: ft_forward (d_img -> d_map) followed by ft_peaks
 * on d_map, with the same arguments, layouts, rules and results (d_map holds
 * the map afterwards).  Where step 4 runs the fixed-length FP32 kernel on the
 * caller's stream (n_intercept with a fixed-length schedule, FP32 precision, no
 * lanes) and ft_peaks' cost model prefers the pass from tile maxima, step 4 also
 * writes the maximum of |P| of every 256-cell tile of its output and the
 * peak pass reads only the tiles whose maximum can reach the top_k: a peak
 * never exceeds its tile's maximum, so once top_k peaks are known, tiles below
 * the top_k-th value cannot contribute; the list is the same as ft_peaks'
 * (Sec. 4.4; checked equal element by element).  4 launches then (5 in the
 * inverse space), else those of ft_forward and ft_peaks.  threshold must not be
 * NaN (FT_ERR_INVALID_ARG, as for ft_peaks). */
ft_status ft_detect(ft_plan plan, const float* d_img, float* d_map, int batch, int top_k, float threshold,
                    ft_peak* d_out, int32_t* d_count, void* stream);

/* ft_detect over nb consecutive batches of `batch` images each, enqueued on
 * `stream` as one pipeline: batch j reads its images from d_imgs[j] (a HOST
 * array of nb device pointers, each to [batch][H][W] FP32, 8-byte aligned) and
 * writes its top_k records per image to d_out + j * batch * top_k and its counts
 * to d_count + j * batch (device, caller-owned, nb * batch * top_k records and
 * nb * batch counts).  d_map ([batch][H'][S]) is scratch shared by the batches
 * and holds the last batch's maps afterwards.  The records and counts equal
 * those of nb ft_detect calls (Sec. 3.1 steps 1-4 and the peak detection of
 * Sec. 4.4 per batch).  Where ft_detect takes the peak pass from tile maxima
 * and the plan launches its fixed-length kernels with programmatic dependent
 * launch (the default; FT_PDL=0 at plan creation turns it off), step 1 of
 * batch j + 1 runs beside the peak pass of batch j: it reads only its images
 * and writes only the plan's workspace, and it completes only after that pass
 * has, so the rest of batch j + 1 is ordered after batch j.  The images must not
 * overlap d_out, d_count or d_map.  Otherwise the batches run as nb ft_detect
 * calls.  Errors as for ft_detect (FT_ERR_INVALID_ARG for a NULL or misaligned
 * pointer in d_imgs or nb < 0); nb or batch 0 is a no-op.  4 launches per batch
 * on the pipelined path. */
ft_status ft_detect_batches(ft_plan plan, const float* const* d_imgs, int nb, int batch, float* d_map, int top_k,
                            float threshold, ft_peak* d_out, int32_t* d_count, void* stream);

/* Loss for fitting by gradient through ft_backward (the paper fits nothing by
 * gradient; this is the loss of the differentiable workload): with
 * r = |d_map| * scale - d_target elementwise,
 *   d_loss[b]     = mean over the H' x S cells of image b of r^2        ([batch], FP32)
 *   d_grad_map    = d(mean of r^2 over all batch x H' x S cells) / d map
 *                 = 2 r scale sign(map) / (batch H' S), sign(0) = 0
 * d_target has the map's layout.  d_grad_map may be NULL (loss only).  The
 * per-image sums are accumulated in a fixed order (FP32 with compensated
 * summation), so repeated calls give identical results. */
ft_status ft_abs_mse_grad(ft_plan plan, const float* d_map, const float* d_target, int batch, float scale,
                          float* d_loss, float* d_grad_map, void* stream);

/* The same loss and, instead of its map gradient, the gradient with respect to
 * the images: ft_abs_mse_grad followed by ft_backward in one call, with the
 * map gradient computed inside the first adjoint kernel as the map and target
 * columns are loaded, so it is never written to or read back from memory.
 * d_grad_img: [batch][H][W] FP32 (device, caller-owned).  The per-image sums
 * are deterministic but summed in another order than ft_abs_mse_grad's (the
 * losses agree to FP32 rounding).  Lengths n_intercept without a fixed-length
 * kernel go through a plan-owned map gradient instead (same results). */
ft_status ft_abs_mse_backward(ft_plan plan, const float* d_map, const float* d_target, int batch, float scale,
                              float* d_loss, float* d_grad_img, void* stream);

/* End-to-end detection from host memory: copies h_img ([batch][H][W]) to a
 * plan-owned device buffer, runs ft_detect (ft_forward and ft_peaks), copies the peaks and
 * counts back to h_out ([batch][top_k]) and h_count ([batch]) and synchronises
 * `stream` before returning.  The batch is processed in chunks of 8 images: a
 * plan-owned copy stream uploads the next chunk while `stream` transforms the
 * current one (pinned h_img lets the copies run asynchronously). */
ft_status ft_detect_host(ft_plan plan, const float* h_img, int batch, int top_k, float threshold,
                         ft_peak* h_out, int32_t* h_count, void* stream);

/* Peak detection without any device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory when they detect peaks: code recording work into a
 * CUDA graph by stream capture (allocation cannot be captured), services that
 * reserve their device memory at start-up and allocate nothing afterwards, and
 * hosts whose device memory belongs to another allocator.
 *
 * Same result as ft_peaks on |d_map| ([batch][n_intercept][n_slope], FP32),
 * written to d_out ([batch][top_k]) and d_count ([batch]), but no plan is
 * needed and nothing is allocated: the per-tile keys go to one fixed array of
 * FT_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that loads
 * libfunnel.so holds until the process exits.  A call needs at most
 * batch x ceil(n_intercept/32) x ceil(n_slope/64) x min(top_k, 512) x 8 bytes
 * plus 8 bytes per map (an upper bound for both tile kinds: maps with
 * n_slope % 128 == 0 and n_intercept % 32 == 0 use tiles of 32 or 64 x 128
 * cells keeping min(top_k, 32 x rows) keys each, i.e. at most half of it;
 * 64 maps of 1024 x 1024 with top_k = 32 use 2 MiB).  A call whose keys would
 * not fit returns FT_ERR_UNSUPPORTED_SIZE and ft_last_error() says why.
 *
 * The first call in a CUDA context looks up the array's device address in that
 * context (under a lock; again after cudaDeviceReset or in another context on
 * the same device, since the address belongs to the context); make that first
 * call before any stream capture.  Later calls issue only stream work
 * (a cudaMemsetAsync and two kernel launches).  All calls share the one array,
 * so calls whose work overlaps on the GPU (other streams, other threads) race
 * on it; calls in order on one stream are safe.
 * n_intercept, n_slope >= 2; 1 <= top_k <= FT_MAX_TOPK; threshold not NaN. */
#define FT_NOALLOC_SCRATCH_BYTES (16u << 20)
ft_status ft_peaks_noalloc(const float* d_map, int n_intercept, int n_slope, int batch, int top_k,
                           float threshold, ft_peak* d_out, int32_t* d_count, void* stream);

/* Kernel variants of a plan, the autotuner's knob (results are identical up to
 * FP32 rounding order): 0 = the fixed-length register-resident kernels where
 * the length has a schedule (the default), generic shared-memory kernels
 * elsewhere; 1..4 = the generic kernels everywhere with the largest column /
 * row blocks (1), half-size column blocks (2), half-size row blocks (3), both
 * halved (4).  FT_FORCE_GENERIC=1 in the environment at plan creation selects 1. */
int ft_plan_variant_count(ft_plan plan);
ft_status ft_plan_set_variant(ft_plan plan, int variant);
int ft_plan_get_variant(ft_plan plan);

/* ------------------------------------------------------------------------
 * Mixed-size batches (the paper's Sec. I remark that rows and columns are
 * independent, taken across images of uneven sizes).  A batch of n images of
 * sizes H[i] x W[i] (maps n_intercept = H[i], n_slope = W[i]) fixes a packed
 * layout: the caller stores the images back to back in the order
 * ft_batch_layout reports (order[j] = the caller's index of packed image j,
 * img_off[j] / map_off[j] = its element offset in the packed image / map
 * buffers, totals = {image elements, map elements}); peaks are written as
 * [n][top_k] rows and counts as [n] in the same packed order.  Equal shapes are
 * contiguous, largest first.
 *
 * Images whose sides both have a fixed-length schedule up to 2048 (128, 192,
 * 256, 384, 512, 768, 1024, 1536, 2048), with the linear or cubic interpolator,
 * run in the grouped kernels: one persistent launch per stage over all of them
 * (step 1; steps 2-3; step 4 with the maxima of |P| per 256-cell tile; the peak
 * pass from those maxima), each block taking (image, block) items from a device
 * work queue, largest images first, and running the fixed-length code of the
 * item's length; 4 launches (3 with top_k = 0) whatever the number of shapes.
 * Every other shape group keeps a plan of its own (one per shape) whose
 * ft_detect (ft_forward when top_k = 0) runs on one of up to 8 side streams
 * forked from and joined back into `stream`.  Results are those of per-image
 * plans (the same FFT arithmetic, bit for bit; the same peak lists).
 *   FT_BATCH_GRAPH: capture the whole sequence once into a CUDA graph (after an
 *     uncaptured run that allocates every workspace and synchronises `stream`)
 *     and replay it while all arguments stay the same; `stream` must not be the
 *     legacy default stream.
 *   FT_BATCH_TUNE: before running, time on the caller's buffers (synchronous)
 *     every combination of the grouped kernels' threads per block (step 1: 256
 *     or 512; steps 2-3: 128 or 256; step 4: 256 or 512 -- which fix the
 *     transforms per block of every length and the tile shape of the peak pass)
 *     and every kernel variant of the other groups' plans (ft_plan_set_variant),
 *     and keep the fastest; with a tune_cache path the choices are merged into
 *     that JSON file (keys "GPU name|HxW|interp" for the plans, "GPU
 *     name|batch|interp|shape digest" for the grouped kernels) and
 *     ft_batch_create applies cached choices.
 * The batch owns its plans, workspaces, streams and graph; one batch may be
 * used by one host thread at a time. */
typedef struct ft_batch_s* ft_batch;
#define FT_BATCH_GRAPH 1
#define FT_BATCH_TUNE 2
ft_status ft_batch_create(ft_batch* out, int n, const int32_t* H, const int32_t* W, int interp,
                          const char* tune_cache);
ft_status ft_batch_destroy(ft_batch batch);
ft_status ft_batch_layout(ft_batch batch, int32_t* order, int64_t* img_off, int64_t* map_off,
                          int64_t* totals);
int ft_batch_group_count(ft_batch batch);
/* info = {H, W, first packed position, count, variant} of group g; variant is
 * -1 for groups in the grouped kernels */
ft_status ft_batch_group_info(ft_batch batch, int g, int32_t* info);
/* mean ms of one tuned forward (+ peaks) of group g alone, -1 before tuning and
 * for groups in the grouped kernels */
float ft_batch_group_tuned_ms(ft_batch batch, int g);
/* info[6] = {images in the grouped kernels, shape groups on plans of their own,
 * threads per block of step 1, of steps 2-3, of step 4 (the grouped kernels),
 * kernel launches of one ft_batch_run with top_k > 0} */
ft_status ft_batch_config(ft_batch batch, int32_t* info);
/* Threads per block of the grouped kernels (256 or 512; 128 or 256; 256 or 512;
 * FT_ERR_INVALID_ARG otherwise).  Changes later runs (the graph is recaptured). */
ft_status ft_batch_set_config(ft_batch batch, int r2c_threads, int rows_threads, int c2r_threads);
/* The autotuner's measurements of the grouped kernels: ms[c] (c < n, at most
 * 8) = mean ms of one run with step 1 threads {256, 512}[c >> 2 & 1], steps
 * 2-3 {128, 256}[c >> 1 & 1], step 4 {256, 512}[c & 1]; -1 before tuning.
 * Returns 8. */
int ft_batch_tune_ms(ft_batch batch, float* ms, int n);
/* Kernel launches of one ft_batch_run with this top_k (0 for an invalid one). */
int ft_batch_launches(ft_batch batch, int top_k);
ft_status ft_batch_run(ft_batch batch, const float* d_imgs, float* d_maps, int top_k, float threshold,
                       ft_peak* d_out, int32_t* d_count, void* stream, int flags);

/* ------------------------------------------------------------------------
 * Split-precision tensor-core transforms (the DFT-by-GEMM variant of the FFT
 * stages).  FT_PRECISION_FP32 is the FFT path; the other two evaluate DFTs as
 * GEMMs on the sm_103a tensor cores (tcgen05.mma, FP32 accumulation in tensor
 * memory) with every FP32 operand split into a high and a low 16-bit part,
 * D = Ahi Bhi + Ahi Blo + Alo Bhi. */
typedef enum {
    FT_PRECISION_FP32 = 0,
    FT_PRECISION_BF16X3 = 1,     /* BF16 hi + lo, 3 products */
    FT_PRECISION_FP16X3 = 2,     /* FP16 hi + lo, 3 products */
    FT_PRECISION_BF16X6 = 3      /* BF16 hi + mid + lo, 6 products (all of order <= 2) */
} ft_precision;

/* Batched 64-point complex DFT y[v][k] = sum_n x[v][n] exp(sign 2 pi i k n / 64)
 * (sign = +1 or -1) for v < nvec, x and y [nvec][64] complex FP32 (interleaved,
 * 8-byte aligned, device).  precision: FT_PRECISION_BF16X3 or _FP16X3.  d_err:
 * a device uint32 that gets bit 0 set if a tensor-core wait timed out (the
 * outputs of that block are then NaN); the caller clears it.  This is the
 * building block of the split-precision FFT stages and their self-check. */
ft_status ft_tc_dft64(const void* d_x, void* d_y, int nvec, int sign, int precision, uint32_t* d_err,
                      void* stream);

/* Arithmetic of the length-4096 Fourier transforms of ft_forward (Sec. 3.1:
 * step 1 along y, eq. (16); step 3 along x', eq. (13); step 4 along omega_2,
 * eq. (19)).  FT_PRECISION_FP32 (the default) is the FP32 FFT.  The split
 * variants evaluate every transform of length 4096 as a four-step DFT,
 * 4096 = 64 x 64: two split-precision GEMMs (the 64-point DFT matrix against
 * 64 rows of gathered or twiddled values) with FP32 twiddles in between, in one
 * persistent kernel per step that keeps the DFT matrix in shared memory: steps
 * 2-3 when n_slope = 4096 (the NVMT gather writes the first GEMM's operand; not
 * with the band-limited interpolator), steps 1 and 4 when n_intercept = 4096
 * (two image or map columns per complex transform).  Transforms of other
 * lengths, the peaks and ft_backward stay FP32.  Returns
 * FT_ERR_UNSUPPORTED_SIZE for a split precision when the plan has no such
 * transform (the plan keeps its previous precision); FT_ERR_INVALID_ARG for an
 * unknown value.  Changes the result of later calls only. */
ft_status ft_plan_set_precision(ft_plan plan, int precision);
int ft_plan_get_precision(ft_plan plan);

/* Error flags of the plan's device-side waits, each bounded by
 * ft_plan_get_wait_cycles SM cycles (about 2 s by default).  Bit 0: a wait for
 * the tensor cores timed out; the row group that gave up waits for its own
 * issued MMAs with the default bound, frees its tensor memory with the rest of
 * its block and stops, so the rows it had not finished are left incomplete.
 * Bit 1: a wait of the FP32 row kernel (steps 2-3) for the bulk copies that
 * stage its spectrum rows timed out; the block waits for its copies in flight
 * with the default bound and returns without writing its rows.  Bit 2: a wait
 * of the inverse column kernel (step 4) for the tensor copies that stage its
 * Hermitian half columns timed out; bit 3: the same for the forward column
 * kernel (step 1) and its image columns, or for the first kernel of
 * ft_abs_mse_backward and its map columns.  Those blocks likewise drain their
 * copies in flight and return without writing.  The CUDA context stays usable
 * in every case.  Waits for all work on the plan's device,
 * copies the flags to *flags (host) and clears them; returns FT_ERR_TIMEOUT
 * when a bit was set (ft_last_error() says which), FT_OK otherwise. */
ft_status ft_plan_tc_errors(ft_plan plan, uint32_t* flags);

/* Bound, in SM cycles, of every device-side wait of the plan's kernels (the
 * tensor-core kernels for their GEMMs, the FP32 row and column kernels for
 * their bulk and tensor copies; FT_WAIT_CYCLES_DEFAULT, about 2 s at 2 GHz, after creation).
 * The limit is checked before each try, so 0 makes every such wait give up at
 * once: a test setting that runs the timeout path (flag, drain, free, stop)
 * without any GPU fault.  cycles < 0 is FT_ERR_INVALID_ARG.  Changes later
 * calls only. */
#define FT_WAIT_CYCLES_DEFAULT 4000000000ll
ft_status ft_plan_set_wait_cycles(ft_plan plan, int64_t cycles);
int64_t ft_plan_get_wait_cycles(ft_plan plan);

/* Failure injection for tests of the error paths: the next `count` device
 * allocations of this plan's workspace or host-path buffers fail as an
 * out-of-memory cudaMalloc would (the call returns FT_ERR_OOM, ft_last_error()
 * names the buffer, nothing is launched); count = 0 clears it.  The plan stays
 * usable: the next call allocates again. */
ft_status ft_plan_inject_alloc_failures(ft_plan plan, int count);

/* Line verification (Sec. 4.5, steps 1-4) of detected peaks.  For peak j of
 * image b (d_peaks[b * top_k + j], j < d_count[b], as written by ft_peaks on
 * this plan's maps) the candidate line is read from the peak's map cell by
 * eqs. (22)-(23) (regular space) or (24)-(25) (inverse space); a band of
 * 2 * half_width + 1 pixels (half_width 1..3: the paper's 3 to 7) centred on
 * the line is cut from the original image d_img (device, [batch][H][W] FP32,
 * the forward's input) and integrated along the line's length: every image
 * column (regular space; image row in the inverse space) gives one sample per
 * offset d = -h..h at the line's centre row + d, linearly interpolated between
 * the two nearest rows, counted where both rows are inside the image.
 * Outputs (device): d_profile[b][j][2h+1] = mean sample per offset,
 * d_length[b][j] = samples on the centre line, d_verdict[b][j] = 1 when
 * d_length >= min_length and max(|p[0] - (p[-h] + p[h]) / 2|, |p[h] - p[-h]| / 2)
 * >= min_contrast (ridge or step edge present), 0 when not, -1 for j >=
 * d_count[b] (profile zeros).  The decision rule and the band geometry are
 * readings of the paper's steps 2-4.  Stream-ordered, no allocation.
 * FT_ERR_INVALID_ARG for null pointers, top_k outside 1..FT_MAX_TOPK or
 * half_width outside 1..3. */
ft_status ft_verify(ft_plan plan, const float* d_img, const ft_peak* d_peaks, const int32_t* d_count, int batch,
                    int top_k, int half_width, float min_contrast, int32_t min_length, float* d_profile,
                    int32_t* d_length, int32_t* d_verdict, void* stream);

/* Bytes of plan-owned device workspace that a call with this batch needs. */
size_t ft_workspace_bytes(ft_plan plan, int batch);

/* Number of kernel launches ft_forward / ft_peaks issue for a call with this
 * batch.  With FT_LANES=2 in the environment at plan creation, a batch of 4 or
 * more images is split over 2 plan-owned streams forked from and joined back
 * into the caller's stream (same kernels, same results, kernels of the two
 * halves overlapping); by default everything runs on the caller's stream. */
int ft_forward_launches(ft_plan plan, int batch);
int ft_peaks_launches(ft_plan plan, int batch);
/* The same for ft_detect with this batch and top_k (0 for an invalid top_k). */
int ft_detect_launches(ft_plan plan, int batch, int top_k);

/* Kernel identifiers of the per-launch timing below. */
typedef enum {
    FT_KERNEL_COL_R2C = 0,         /* step 1 (and the transpose of step 4) */
    FT_KERNEL_NVMT_ROWS = 1,       /* steps 2-3 */
    FT_KERNEL_COL_C2R = 2,         /* step 4 (and the transpose of step 1) */
    FT_KERNEL_PEAK_TILES = 3,      /* Sec. 4.4, local maxima per tile */
    FT_KERNEL_PEAK_SELECT = 4,     /* Sec. 4.4, top_k per image */
    FT_KERNEL_NVMT_ROWS_ADJ = 5,   /* transpose of steps 2-3 */
    FT_KERNEL_LOSS = 6,            /* ft_abs_mse_grad */
    FT_KERNEL_VERIFY = 7,          /* ft_verify, Sec. 4.5 */
    FT_KERNEL_PEAK_SPARSE = 8,     /* Sec. 4.4 from tile maxima (ft_peaks, ft_detect) */
    FT_KERNEL_TILE_MAX = 9,        /* tile maxima of a given map (ft_peaks) */
    FT_KERNEL_COUNT = 10
} ft_kernel_id;

/* Per-launch timing (a measurement aid, off by default).  While enabled, every
 * kernel launch of this plan is bracketed by two CUDA events recorded on the
 * launching stream.  ft_profile_read synchronises those events, adds each
 * launch's elapsed time to total_ms[id] and its count to launches[id] for
 * id < n (arrays of n entries, zeroed first), and forgets the records. */
ft_status ft_profile_enable(ft_plan plan, int enable);
ft_status ft_profile_read(ft_plan plan, double* total_ms, int32_t* launches, int n);
const char* ft_kernel_name(int id);

/* FP32 FMA throughput probe (a measurement aid for the ALU roofline; no part
 * of the transform): `blocks` blocks of 256 threads, each thread running 8
 * independent FMA chains for `iters` rounds, one float per thread written to
 * d_out (device, blocks x 256 floats).  FLOPs of one call:
 * blocks x 256 x iters x 16.  Time it with CUDA events on `stream`. */
ft_status ft_fma_probe(float* d_out, int blocks, int iters, void* stream);

/* Bounds-checked debug build (libfunnel_debug.so, compiled with FT_DEBUG): the
 * device checks every gather / scatter index of the fixed-length transform
 * kernels and the peak pass; an index out of range is skipped (a load reads 0)
 * and sets a bit in a flag word: 1 step-1 loads, 2 step-1 stores, 4 step-4
 * staging, 8 step-4 stores, 16 NVMT taps, 32 FFT exchange slots, 64 NVMT
 * transpose, 128 peak staging.  ft_debug_flags waits for the device, returns
 * the bits recorded since the last call in *flags and clears them (0 in the
 * normal build, where the checks do not exist).  ft_debug_build returns 1 for
 * the debug build, 0 otherwise. */
ft_status ft_debug_flags(uint32_t* flags);
int ft_debug_build(void);

/* Static text for a status; never NULL. */
const char* ft_status_string(ft_status status);

/* Text of the last error recorded by a call in this thread: the CUDA error of
 * an FT_ERR_CUDA, or the reason ft_peaks_noalloc rejected a size ("" if none). */
const char* ft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FUNNEL_H */
