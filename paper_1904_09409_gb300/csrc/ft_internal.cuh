// Internal declarations of libfunnel: plan object, FFT descriptors, complex
// helpers, the shared-memory mixed-radix FFT used by every transform kernel,
// and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "funnel.h"

#define FT_MAX_STAGES 16
#define FT_THREADS 256
// a wait for the tensor cores that has not completed after this many SM cycles
// (about 2 s) gives up (ft_plan_set_wait_cycles changes it per plan)
#define FT_WAIT_CYCLES 4000000000ll

// ------------------------------------------------ bounds-checked debug build
// Compiled with -DFT_DEBUG (libfunnel_debug.so, which the Python binding loads
// when FT_DEBUG=1), every gather / scatter index of the kernels passes through
// FT_IN(index, size, code): an index outside [0, size) sets the bit `code` in
// the translation unit's flag word and the access is skipped (a load reads 0).
// Nothing traps; ft_debug_flags() reads and clears the words of all units.  In
// the normal build FT_IN is the constant true and the checks compile away.
#define FT_DBG_R2C_LOAD 1u        // step 1: image rows / columns read
#define FT_DBG_R2C_STORE 2u       // step 1: half-spectrum rows written
#define FT_DBG_C2R_STAGE 4u       // step 4: Hermitian rows staged / gathered
#define FT_DBG_C2R_STORE 8u       // step 4: map rows, tile maxima written
#define FT_DBG_NVMT_GATHER 16u    // step 2: interpolation taps of a staged row
#define FT_DBG_FFT_SLOT 32u       // exchange slots of the register FFT
#define FT_DBG_NVMT_ADJ 64u       // transpose of step 2: samples gathered back
#define FT_DBG_PEAK_STAGE 128u    // peak pass: staged tile cells
#ifdef FT_DEBUG
static __device__ unsigned g_ft_debug;
__device__ __forceinline__ bool ft_in_range(long long i, long long n, unsigned code) {
    if (i >= 0 && i < n) return true;
    atomicOr(&g_ft_debug, code);
    return false;
}
#define FT_IN(i, n, code) ft_in_range((long long)(i), (long long)(n), (code))
#define FT_DEBUG_READER(name)                                                 \
    unsigned name() {                                                         \
        unsigned v = 0, z = 0;                                                \
        if (cudaMemcpyFromSymbol(&v, g_ft_debug, sizeof(v)) != cudaSuccess) return 0x80000000u; \
        cudaMemcpyToSymbol(g_ft_debug, &z, sizeof(z));                        \
        return v;                                                             \
    }
#else
#define FT_IN(i, n, code) true
#define FT_DEBUG_READER(name) \
    unsigned name() { return 0u; }
#endif
// the flag words of the units with checks (host; the device must be idle)
unsigned ft_debug_read_fast();
unsigned ft_debug_read_peak_sparse();

// One FFT length N = 2^a 3^b: its radix sequence and twiddle table
// tw[t] = exp(-2 pi i t / N), t in [0, N), rounded to FP32 from FP64 values.
struct FftLen {
    int N;
    int nst;
    int radix[FT_MAX_STAGES];
    const float2* tw;
    const float2* stw;      // per-pass twiddles of the fixed-length kernels (NULL: generic path)
};

// ------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by (SIGN * i): SIGN = +1 -> i*a, SIGN = -1 -> -i*a
template <int SIGN>
__device__ __forceinline__ float2 cmul_si(float2 a) {
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Twiddle exp(SIGN * 2 pi i t / N) from the table of exp(-2 pi i t / N).
template <int SIGN>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int t) {
    float2 w = __ldg(tw + t);
    return SIGN > 0 ? make_float2(w.x, -w.y) : w;
}

// ------------------------------------------- programmatic dependent launch
// A kernel of the forward chain (steps 1, 2-3 and 4, the peak pass) may be
// launched while its predecessor on the stream is still running (its blocks are
// placed as the predecessor's last blocks retire); pdl_wait() blocks until the
// predecessor has completed and its writes are visible, and is a no-op for a
// kernel launched without the attribute.  Every such kernel calls it before its
// first read or write of device memory.  pdl_trigger() lets the successor be
// launched early (steps 1-4 call it when their blocks start, the peak pass
// after its wait).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// launch kernel k (grid g, block b, sm bytes of dynamic shared memory) on st,
// with programmatic stream serialisation when pdl is set
template <typename... KArgs, typename... Args>
static cudaError_t launch_maybe_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st, bool pdl,
                                    Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// ----------------------------------------------------- NVMT index helpers
__device__ __forceinline__ int floor_div(int a, int b) {   // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int ceil_div(int a, int b) {    // b > 0
    int q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

// Keys' cubic convolution kernel with a = -0.5.
__device__ __forceinline__ float keys_w(float s) {
    const float a = -0.5f;
    s = fabsf(s);
    if (s <= 1.f) return ((a + 2.f) * s - (a + 3.f)) * s * s + 1.f;
    if (s < 2.f) return ((a * s - 5.f * a) * s + 8.f * a) * s - 4.f * a;
    return 0.f;
}

// Weight of tap offset d (tap = floor + d) at fraction fr: linear uses d = 0, 1;
// cubic d = -1 .. 2.
__device__ __forceinline__ float tap_weight(int interp, int d, float fr) {
    if (interp == FT_INTERP_LINEAR) return d == 0 ? 1.f - fr : fr;
    return keys_w(fr - (float)d);
}

// ---------------------------------------------------------- radix-R kernels
// y_k = sum_q u_q exp(SIGN 2 pi i q k / R), in place.
template <int R, int SIGN>
struct Dft;

template <int SIGN>
struct Dft<2, SIGN> {
    __device__ __forceinline__ static void run(float2* u) {
        float2 a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    }
};

template <int SIGN>
struct Dft<3, SIGN> {
    __device__ __forceinline__ static void run(float2* u) {
        const float h = 0.86602540378443864676f;   // sqrt(3)/2
        float2 s = cadd(u[1], u[2]);
        float2 d = csub(u[1], u[2]);
        float2 y0 = cadd(u[0], s);
        float2 t1 = make_float2(u[0].x - 0.5f * s.x, u[0].y - 0.5f * s.y);
        float2 t2 = cscale(cmul_si<SIGN>(d), h);
        u[0] = y0;
        u[1] = cadd(t1, t2);
        u[2] = csub(t1, t2);
    }
};

template <int SIGN>
struct Dft<4, SIGN> {
    __device__ __forceinline__ static void run(float2* u) {
        float2 a = cadd(u[0], u[2]), b = csub(u[0], u[2]);
        float2 c = cadd(u[1], u[3]), d = cmul_si<SIGN>(csub(u[1], u[3]));
        u[0] = cadd(a, c);
        u[2] = csub(a, c);
        u[1] = cadd(b, d);
        u[3] = csub(b, d);
    }
};

template <int SIGN>
struct Dft<8, SIGN> {
    __device__ __forceinline__ static void run(float2* u) {
        const float r = 0.70710678118654752440f;   // sqrt(2)/2
        float2 e[4] = {u[0], u[2], u[4], u[6]};
        float2 o[4] = {u[1], u[3], u[5], u[7]};
        Dft<4, SIGN>::run(e);
        Dft<4, SIGN>::run(o);
        // w8^k = exp(SIGN 2 pi i k / 8)
        float2 o1 = make_float2(r * (o[1].x - SIGN * o[1].y), r * (o[1].y + SIGN * o[1].x));
        float2 o2 = cmul_si<SIGN>(o[2]);
        float2 o3 = make_float2(r * (-o[3].x - SIGN * o[3].y), r * (-o[3].y + SIGN * o[3].x));
        u[0] = cadd(e[0], o[0]);
        u[4] = csub(e[0], o[0]);
        u[1] = cadd(e[1], o1);
        u[5] = csub(e[1], o1);
        u[2] = cadd(e[2], o2);
        u[6] = csub(e[2], o2);
        u[3] = cadd(e[3], o3);
        u[7] = csub(e[3], o3);
    }
};

// ------------------------------------------------- Stockham stage (autosort)
// B transforms of length N interleaved in shared memory as x[n * B + f].
// Stage with radix R after sub-transforms of length p: for i in [0, N/R),
// k = i mod p, inputs x[i + q N/R] twiddled by exp(SIGN 2 pi i q k / (p R)),
// radix-R DFT, outputs y[(i - k) R + k + q p].
template <int R, int SIGN>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ x, float2* __restrict__ y,
                                          int N, int logB, int p, const float2* __restrict__ tw) {
    const int B = 1 << logB;
    const int NR = N / R;
    const int tws = N / (p * R);
    const int total = NR << logB;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int f = idx & (B - 1);
        const int i = idx >> logB;
        const int k = i % p;
        float2 u[R];
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = x[((i + q * NR) << logB) + f];
        if (p > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) u[q] = cmul(u[q], twiddle<SIGN>(tw, q * k * tws));
        }
        Dft<R, SIGN>::run(u);
        const int j = (i - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) y[((j + q * p) << logB) + f] = u[q];
    }
}

// Full transform of the B interleaved sequences in `a` (length N each) using
// `b` as the ping-pong buffer.  Returns the buffer that holds the result.
// Must be called by every thread of the block; ends with __syncthreads().
template <int SIGN>
__device__ float2* cta_fft(float2* a, float2* b, const FftLen& L, int logB) {
    int p = 1;
    for (int s = 0; s < L.nst; ++s) {
        const int R = L.radix[s];
        switch (R) {
            case 2: fft_stage<2, SIGN>(a, b, L.N, logB, p, L.tw); break;
            case 3: fft_stage<3, SIGN>(a, b, L.N, logB, p, L.tw); break;
            case 4: fft_stage<4, SIGN>(a, b, L.N, logB, p, L.tw); break;
            default: fft_stage<8, SIGN>(a, b, L.N, logB, p, L.tw); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        p *= R;
    }
    return a;
}

// -------------------------------------------------------------- plan object
struct ft_plan_s {
    int H, W, S, Hp, L, interp, top;   // the transform's own sizes (transposed for the inverse space)
    int space;              // FT_SPACE_REGULAR or FT_SPACE_INVERSE
    int img_H, img_W;       // the caller's image sizes
    int device;
    FftLen fy;              // length H' (steps 1 and 4)
    FftLen fx;              // length S  (step 3)
    float2* d_tw;           // both twiddle tables in one allocation
    // workspace: spectrum / G rows [batch][L][S] complex, then peak keys
    void* d_ws;
    size_t ws_bytes;
    // host-path buffers of ft_detect_host
    float* d_img_host;
    size_t img_host_bytes;
    float* d_map_host;
    size_t map_host_bytes;
    ft_peak* d_peaks_host;
    int32_t* d_count_host;
    size_t peaks_host_bytes;
    // launch shapes
    int col_logB_y;         // transforms per CTA (log2) for length H' (generic kernels)
    int row_logB_x;         // rows per CTA (log2) for length S (generic kernels)
    int col_logB_max, row_logB_max;  // the largest that fit the shared-memory budget
    int use_fast_y, use_fast_x;      // fixed-length kernels in use for H' / S
    int variant;            // see ft_plan_set_variant
    int peak_mode;          // peak pass: 0 = the faster one by the cost model, 1 = from tile maxima, 2 = per-tile keys
    int num_sms;            // multiprocessors of the plan's device
    int pdl;                // programmatic dependent launch in the forward chain (FT_PDL=0: off)
    int precision;          // ft_precision of step 3 (ft_plan_set_precision)
    unsigned* d_tc_err;     // error flags of the tensor-core kernels (allocated with the first split precision)
    long long tc_wait;      // bound of every tensor-core wait in SM cycles (ft_plan_set_wait_cycles)
    int alloc_failures;     // device allocations still to fail (ft_plan_inject_alloc_failures)
    // band-limited (chirp-z) interpolator: lengths W and M >= W + S, chirp tables
    FftLen fw, fm;
    float2* d_chirp;        // [L][W+1] pre-chirps, [L][S] post-chirps, [L][M] chirp spectra
    // lanes: the batch split over FT_LANES plan-owned streams forked from the caller's
    cudaStream_t lane_streams[2];
    cudaEvent_t lane_fork, lane_join[2];
    int lanes;
    // ft_detect_host pipeline: a copy stream and one event per chunk
    cudaStream_t copy_stream;
    std::vector<cudaEvent_t> chunk_events;
    cudaEvent_t start_event;
    // per-launch timing (ft_profile_enable / ft_profile_read)
    int prof_on;
    size_t prof_used;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<int> prof_ids;      // kernel id of each recorded launch (events 2i, 2i+1)
};

// Record an error text for ft_last_error() in the calling thread and return the
// status (FT_ERR_CUDA for the CUDA variant).
ft_status ft_record_cuda(cudaError_t e, const char* where);
ft_status ft_record_error(ft_status s, const char* text);

// -------------------------------------------------------- kernel launchers
// All return the cudaError_t of the launch.

// Step 1 (and the transpose of step 4): real columns -> half spectra.
// in: [batch] x rows_in x ncols (pitch in_pitch floats, image stride in_img),
// zero-expanded to N rows with the first input row at expanded row `row0`.
// out[l][c] (complex, pitch out_pitch, image stride out_img) for l in [0, N/2],
// scaled by end_scale (l = 0, N/2) or mid_scale (0 < l < N/2).
cudaError_t launch_col_r2c(const float* in, int rows_in, int ncols, int in_pitch, size_t in_img,
                           int row0, const FftLen& f, int logB, float2* out, int out_pitch,
                           size_t out_img, float end_scale, float mid_scale, int batch,
                           cudaStream_t st);

// Step 4 (and the transpose of step 1): half spectra -> real columns.
// in[l][c] (complex, pitch in_pitch, image stride in_img) for l in [0, N/2]; the
// end bins enter through their real part, interior bins are scaled by mid_scale;
// out rows t in [row0, row0 + rows_out) of the length-N result, times out_scale,
// go to out[(t - row0)][c] (pitch out_pitch floats, image stride out_img).
cudaError_t launch_col_c2r(const float2* in, int ncols, int in_pitch, size_t in_img,
                           const FftLen& f, int logB, float mid_scale, float* out, int row0,
                           int rows_out, int out_pitch, size_t out_img, float out_scale,
                           int batch, cudaStream_t st);

// Steps 2-3 in place on ws rows l in [0, L): gather/interpolate W columns to S
// samples, transform with exp(+j), write S values.  Row 0 becomes zero.
cudaError_t launch_nvmt_rows(float2* ws, int W, int S, int Hp, int L, int interp,
                             const FftLen& fx, int logRB, int batch, cudaStream_t st);

// Transpose of steps 2-3 in place: S values -> transform with exp(-j) ->
// scatter of the interpolation weights gathered back to W columns.
cudaError_t launch_nvmt_rows_adjoint(float2* ws, int W, int S, int Hp, int L, int interp,
                                     const FftLen& fx, int logRB, int batch, cudaStream_t st);

// Peak detection of Sec. 4.4: per-tile strict local maxima -> per-tile best
// keys (launch_peak_tiles), then per-image selection of the top_k keys in order
// (launch_peak_select).  keys must hold peaks_key_bytes() bytes.  bounds holds
// two words per image (the running bound of the top_k-th value and the length
// of the image's appended key list); the sub-batch of images b0.. uses
// keys + b0 * peaks_tile_keys() and bounds + 2 * b0.
cudaError_t launch_peak_tiles(const float* map, int Hp, int S, int batch, int top_k, float threshold,
                              unsigned long long* keys, unsigned* bounds, cudaStream_t st);
// keys per image, and the per-image words inside a key buffer of
// peaks_key_bytes(Hp, S, batch, top_k) bytes
size_t peaks_tile_keys(int Hp, int S, int top_k);
unsigned* peaks_bounds(unsigned long long* keys, int Hp, int S, int batch, int top_k);
cudaError_t launch_peak_select(const unsigned long long* keys, const unsigned* bounds, int Hp, int S, int batch,
                               int top_k, ft_peak* out, int32_t* count, cudaStream_t st);
size_t peaks_key_bytes(int Hp, int S, int batch, int top_k);

// The same detected list from tile maxima of |map| (k_peak_sparse.cu): tmax
// [batch][ceil(Hp / tile_rows)][ceil(S / tile_cols)] float bits of the maximum
// of each tile (the last ones ragged), from step 4 (launch_col_c2r_fast) or
// launch_tile_max; one block per image reads only the tiles that can hold one
// of the top_k peaks.  peak_sparse_fits: the tile shape is usable (tile_cols a
// power of two, tile_rows x tile_cols a multiple of 32) and the pass's shared
// memory fits the current device.
bool peak_sparse_fits(int tile_rows, int tile_cols, int top_k);
cudaError_t launch_peak_sparse(const float* map, const unsigned* tmax, int Hp, int S, int tile_rows, int tile_cols,
                               int batch, int top_k, float threshold, ft_peak* out, int32_t* count, cudaStream_t st,
                               bool pdl = false);
// tile maxima of given maps (map 8-byte aligned) in tiles of tile_max_shape
void tile_max_shape(int* tile_rows, int* tile_cols);
cudaError_t launch_tile_max(const float* map, int Hp, int S, int batch, unsigned* tmax, cudaStream_t st);

// the band-limited NVMT fused with step 3 (k_fourier.cu)
cudaError_t launch_chirp_fft(float2* hc, int L, const FftLen& fm, cudaStream_t st);
cudaError_t launch_nvmt_rows_fourier_adj(float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                         const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                         const float2* chirp_x, const float2* hc, int batch, cudaStream_t st);
cudaError_t launch_nvmt_rows_fourier(float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                     const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                     const float2* chirp_x, const float2* hc, int batch, cudaStream_t st);

// the same on the register-resident FFT (k_fourier_fast.cu) where W = S, M = 2W
// and all three lengths have a schedule (fw, fm, fs with per-pass twiddles);
// cudaErrorNotSupported otherwise
bool fourier_fast_ok(int W, int M, int S);
cudaError_t launch_nvmt_rows_fourier_fast(bool adjoint, float2* ws, int W, int S, int Hp, int L, const FftLen& fw,
                                          const FftLen& fm, const FftLen& fs, const float2* chirp_u,
                                          const float2* chirp_x, const float2* hc, int batch, cudaStream_t st);

// batched 64-point DFT as a split-precision tensor-core GEMM (k_tc.cu);
// fmt 1 = BF16 hi+lo, 0 = FP16 hi+lo; err gets bit 0 set if a wait timed out
cudaError_t launch_tc_dft64(const float2* x, float2* y, int nvec, int sign, int fmt, unsigned* err,
                            cudaStream_t st);
// tables of the tensor-core kernels on the current device (host call, before any capture)
cudaError_t tc_prepare();
// The split-precision four-step DFT of length 4096 (k_tc.cu): steps 2-3 for
// n_slope = 4096, and steps 1 and 4 of the forward path for n_intercept = 4096
// (launch_col_r2c with unit scales, but the image column-major [batch][W][H];
// launch_col_c2r with mid scale 1 and out scale 1/H', but the map written
// column-major [batch][S][H'])
// (prec: FT_PRECISION_BF16X3, _FP16X3 or _BF16X6)
// (wait: the bound of every wait for the tensor cores, in SM cycles)
cudaError_t launch_nvmt_rows_tc4096(float2* ws, int W, int Hp, int L, int interp, int prec, unsigned* err,
                                    long long wait, int batch, cudaStream_t st);
cudaError_t launch_col_r2c_tc4096(const float* img_cm, int H, int W, int row0, float2* ws, int L, int S, int prec,
                                  unsigned* err, long long wait, int batch, cudaStream_t st);
cudaError_t launch_col_c2r_tc4096(const float2* ws, int L, int S, float* map_cm, int prec, unsigned* err,
                                  long long wait, int batch, cudaStream_t st);

// ---------------------------------------------- mixed-size batches (k_batch.cu)
// One image of a mixed-size batch in the grouped kernels: map n_intercept = H,
// n_slope = W; offsets in elements of the packed images / maps, complex
// elements of the batch's spectrum workspace and words of its tile maxima.
struct BatchImg {
    long long img_off, map_off, ws_off, tm_off;
    int H, W;
    int pos;                // packed position (row of the peak records and counts)
    const float2* stw_y;    // per-pass twiddles of length H (steps 1 and 4)
    const float2* stw_x;    // per-pass twiddles of length W (step 3)
};
// lengths the grouped kernels take (every fixed-length schedule up to 2048)
__host__ __device__ constexpr bool batch_len_ok(int n) {
    return n == 128 || n == 192 || n == 256 || n == 384 || n == 512 || n == 768 || n == 1024 || n == 1536 ||
           n == 2048;
}
// blocks of one image per stage for the given threads per block (the stage's
// tuning knob); rows: NVMT + row FFT blocks; cols: column blocks of step 1 / 4
int batch_r2c_blocks(int H, int W, int threads);
int batch_rows_blocks(int H, int W, int threads);
int batch_c2r_blocks(int H, int W, int threads);
// tile shape of step 4's maxima: rows x cols cells, bands x column blocks tiles
void batch_tile_shape(int H, int W, int threads, int* rows, int* cols, int* bands, int* nbx);
bool batch_threads_ok(int stage, int threads);   // stage 0 r2c, 1 rows, 2 c2r
// The four stage kernels, each a persistent loop over a device work queue of
// `items` (image, block) pairs (*queue counts taken items and must be 0 at the
// launch; the peak stage takes one image per item).  grid = 0 picks the
// resident-block count of the device.
cudaError_t launch_batch_r2c(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, const float* in,
                             float2* ws, int threads, int maxH, cudaStream_t st);
cudaError_t launch_batch_rows(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, float2* ws,
                              int interp, int threads, int maxW, cudaStream_t st);
cudaError_t launch_batch_c2r(const BatchImg* imgs, const int2* items, int nitems, unsigned* queue, const float2* ws,
                             float* maps, unsigned* tmax, int threads, int maxH, cudaStream_t st);
cudaError_t launch_batch_peaks(const BatchImg* imgs, int nimg, unsigned* queue, const float* maps, const unsigned* tmax,
                               int c2r_threads, int top_k, float threshold, ft_peak* out, int32_t* count,
                               size_t smem, cudaStream_t st);
size_t batch_peaks_smem(const BatchImg* host_imgs, int nimg, int c2r_threads, int top_k);

// line verification of Sec. 4.5 (k_verify.cu): image element (v, u) of the
// transform's frame at img[v * stride_v + u * stride_u] (image b at b * img_stride)
cudaError_t launch_verify(const float* img, int H, int W, int stride_v, int stride_u, size_t img_stride, int S,
                          int Hp, const ft_peak* peaks, const int32_t* count, int batch, int top_k, int h,
                          float min_contrast, int min_length, float* profile, int32_t* length, int32_t* verdict,
                          cudaStream_t st);

// in[b][R][C] -> out[b][C][R] (k_transpose.cu)
cudaError_t launch_transpose(const float* in, float* out, int R, int C, int batch, cudaStream_t st);

// Loss of the gradient workload and its gradient (k_loss.cu); partial needs
// loss_partial_bytes(batch) bytes of scratch.
cudaError_t launch_abs_mse_grad(const float* map, const float* target, int batch, size_t cells, float scale,
                                float* loss, float* grad, float* partial, cudaStream_t st);
size_t loss_partial_bytes(int batch);
// per-image loss from nblk partials each (fixed order, compensated), divided by cells
cudaError_t launch_loss_finish(const float* partial, int nblk, size_t cells, float* loss, int batch, cudaStream_t st);
