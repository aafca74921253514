// C ABI of libfunnel: plan creation (validation, FP64-derived twiddle tables,
// launch shapes), workspace management and the forward / adjoint / peak /
// host-buffer entry points declared in funnel.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include <stdlib.h>

#include "fft_fast.cuh"

static thread_local char g_last_error[256] = "";

#define FT_DETECT_CHUNK 8   // images per chunk of the ft_detect_host pipeline
#define FT_LANES 2          // streams a large batch is split over (see lanes_fork)

static ft_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return FT_ERR_CUDA;
}

ft_status ft_record_cuda(cudaError_t e, const char* where) { return cuda_fail(e, where); }

ft_status ft_record_error(ft_status s, const char* text) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", text);
    return s;
}

#define FT_CUDA(call, where)                              \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// N = 2^a 3^b with N even?  Fills the radix list (8s, then one 4 or 2, then 3s).
static bool factorize(int N, FftLen* f) {
    if (N < 2 || N > FT_MAX_LENGTH || (N & 1)) return false;
    int m = N, p2 = 0, p3 = 0;
    while (m % 2 == 0) { m /= 2; ++p2; }
    while (m % 3 == 0) { m /= 3; ++p3; }
    if (m != 1) return false;
    int n = 0;
    while (p2 >= 3) { f->radix[n++] = 8; p2 -= 3; }
    if (p2 == 2) f->radix[n++] = 4;
    if (p2 == 1) f->radix[n++] = 2;
    for (int i = 0; i < p3; ++i) f->radix[n++] = 3;
    if (n > FT_MAX_STAGES) return false;
    f->N = N;
    f->nst = n;
    return true;
}

// tw[t] = exp(-2 pi i t / N) in FP64, rounded once to FP32.  The angle is reduced
// to the first octant with exact integer arithmetic before calling cos/sin.
static void twiddles(int N, float2* out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < N; ++t) {
        // 8 t / N = octant + remainder; use symmetries of cos/sin
        long long u = (long long)t * 8;
        int oct = (int)(u / N);
        long long r = u - (long long)oct * N;    // angle = 2 pi (oct N + r) / (8 N)
        double th = two_pi * (double)r / (8.0 * N);
        double c = cos(th), s = sin(th);
        // rotate by oct * 45 degrees exactly via exact pairs
        double cc, ss;
        const double h = 0.70710678118654752440084436210485;
        switch (oct & 7) {
            case 0: cc = c; ss = s; break;
            case 1: cc = h * (c - s); ss = h * (c + s); break;
            case 2: cc = -s; ss = c; break;
            case 3: cc = -h * (c + s); ss = h * (c - s); break;
            case 4: cc = -c; ss = -s; break;
            case 5: cc = -h * (c - s); ss = -h * (c + s); break;
            case 6: cc = s; ss = -c; break;
            default: cc = h * (c + s); ss = -h * (c - s); break;
        }
        out[t] = make_float2((float)cc, (float)(-ss));
    }
}

// ------------------------------------------------------ per-launch timing
static bool prof_begin(ft_plan p, int id, cudaStream_t st) {
    if (!p->prof_on) return false;
    while (p->prof_pool.size() < p->prof_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        p->prof_pool.push_back(e);
    }
    if (cudaEventRecord(p->prof_pool[p->prof_used], st) != cudaSuccess) return false;
    p->prof_ids.push_back(id);
    p->prof_used += 2;
    return true;
}

static void prof_end(ft_plan p, cudaStream_t st) { cudaEventRecord(p->prof_pool[p->prof_used - 1], st); }

#define FT_LAUNCH(p, id, st, call, where)                    \
    do {                                                     \
        const bool pr_ = prof_begin((p), (id), (st));        \
        cudaError_t e_ = (call);                             \
        if (pr_) prof_end((p), (st));                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);  \
    } while (0)

// exp(sign * j * pi * Hp * n^2 / (2 l W)) with the phase reduced exactly:
// pi Hp n^2 / (2 l W) = 2 pi r / (4 l W), r = Hp n^2 mod 4 l W
static float2 chirp(long long n, int Hp, int l, int W, int sign) {
    const long long den = 4ll * l * W;
    long long r = ((long long)Hp * ((n * n) % den)) % den;
    const double th = 6.283185307179586476925286766559 * (double)r / (double)den;
    return make_float2((float)cos(th), (float)(sign * sin(th)));
}

// Chirp tables of the band-limited interpolator (see k_fourier.cu): per row
// l >= 1, pre-chirps exp(+j pi b u^2) (u = -W/2 .. W/2), post-chirps
// exp(+j pi b x'^2) (x' = -S/2 .. S/2-1) and the spectrum of the convolution
// chirp h[j mod M] = exp(-j pi b (j + W/2 - S/2)^2), j = -W .. S-1, b = Hp/(2 l W).
static ft_status build_chirps(ft_plan p) {
    const int W = p->W, S = p->S, L = p->L, M = p->fm.N;
    const size_t nu = (size_t)L * (W + 1), nx = (size_t)L * S, nh = (size_t)L * M;
    std::vector<float2> h(nu + nx + nh, make_float2(0.f, 0.f));
    float2* cu = h.data();
    float2* cx = cu + nu;
    float2* hc = cx + nx;
    for (int l = 1; l < L; ++l) {
        for (int i = 0; i <= W; ++i) cu[(size_t)l * (W + 1) + i] = chirp(i - W / 2, p->Hp, l, W, +1);
        for (int k = 0; k < S; ++k) cx[(size_t)l * S + k] = chirp(k - S / 2, p->Hp, l, W, +1);
        for (int j = -W; j < S; ++j)
            hc[(size_t)l * M + ((j % M) + M) % M] = chirp(j + W / 2 - S / 2, p->Hp, l, W, -1);
    }
    cudaError_t e = cudaMalloc(&p->d_chirp, h.size() * sizeof(float2));
    if (e != cudaSuccess) {
        p->d_chirp = nullptr;
        cuda_fail(e, "cudaMalloc(chirps)");
        return FT_ERR_OOM;
    }
    e = cudaMemcpy(p->d_chirp, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_chirp_fft(p->d_chirp + nu + nx, L, p->fm, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? FT_OK : cuda_fail(e, "chirp tables");
}

// Per-pass twiddles of the fixed-length kernels: for pass s >= 1 with radix R and
// P = product of the earlier radices, row k (stride fs_rs(R, seed)) holds
// exp(-2 pi i q k / (P R)) at column q (full table), or at column j the power
// q = 1 << j for j < fs_nseed(R) (seed table: the row lengths fx, fw, fm), taken
// from the exact-index table tw of length N; padding entries are zero.
static void stage_twiddles(int N, const float2* tw, float2* out, bool seed) {
    for (int s = 1; s < fs_nst(N); ++s) {
        const int R = fs_radix(N, s), P = fs_P(N, s), step = N / (P * R), RS = fs_rs(R, seed);
        const int ncol = seed ? fs_nseed(R) : R;
        float2* o = out + fs_twoff(N, s, seed);
        for (int k = 0; k < P; ++k)
            for (int j = 0; j < RS; ++j)
                o[k * RS + j] = j < ncol ? tw[(seed ? 1 << j : j) * k * step] : make_float2(0.f, 0.f);
    }
}

static int log2_floor(int v) {
    int l = 0;
    while ((2 << l) <= v) ++l;
    return l;
}

static void free_ws(ft_plan p) {
    if (p->d_ws) cudaFree(p->d_ws);
    p->d_ws = nullptr;
    p->ws_bytes = 0;
}

// Grow a plan-owned device buffer to `need` bytes (synchronise, free, allocate).
// While the plan has injected failures left (ft_plan_inject_alloc_failures), an
// allocation fails as cudaMalloc's out-of-memory error would, without calling it.
static ft_status ensure(ft_plan p, void** ptr, size_t* have, size_t need, const char* what) {
    if (need <= *have && *ptr) return FT_OK;
    if (*ptr) {
        cudaDeviceSynchronize();
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaErrorMemoryAllocation;
    if (p->alloc_failures > 0)
        --p->alloc_failures;
    else
        e = cudaMalloc(ptr, need);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cuda_fail(e, what);
        return FT_ERR_OOM;
    }
    *have = need;
    return FT_OK;
}

static size_t spec_bytes(ft_plan p, int batch) { return (size_t)batch * p->L * p->S * sizeof(float2); }
static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
// workspace: [half spectra][transposed image (inverse space only)][aux: peak keys or loss partials]
static size_t tposed_off(ft_plan p, int batch) { return al256(spec_bytes(p, batch)); }
static size_t tposed_bytes(ft_plan p, int batch) {
    return p->space == FT_SPACE_INVERSE ? al256((size_t)batch * p->H * p->W * sizeof(float)) : 0;
}
static size_t aux_off(ft_plan p, int batch) { return tposed_off(p, batch) + tposed_bytes(p, batch); }

// Fixed-length kernels where the length has a schedule, generic ones otherwise.
static cudaError_t col_r2c(ft_plan p, const float* in, int rows_in, int ncols, int in_pitch,
                           size_t in_img, int row0, float2* out, float es, float ms, int batch,
                           cudaStream_t st, bool follows_peak = false) {
    const size_t out_img = (size_t)p->L * p->S;
    if (p->use_fast_y)
        return launch_col_r2c_fast(in, rows_in, ncols, in_pitch, in_img, row0, p->fy, out, p->S, out_img,
                                   es, ms, batch, st, p->pdl, follows_peak, p->d_tc_err, p->tc_wait);
    return launch_col_r2c(in, rows_in, ncols, in_pitch, in_img, row0, p->fy, p->col_logB_y, out, p->S,
                          out_img, es, ms, batch, st);
}

static cudaError_t col_c2r(ft_plan p, const float2* in, int ncols, float mid, float* out, int row0,
                           int rows_out, int out_pitch, size_t out_img, float os, int batch,
                           cudaStream_t st, unsigned* tmax = nullptr) {
    const size_t in_img = (size_t)p->L * p->S;
    if (p->use_fast_y)
        return launch_col_c2r_fast(in, ncols, p->S, in_img, p->fy, mid, out, row0, rows_out, out_pitch,
                                   out_img, os, batch, st, tmax, p->pdl, p->d_tc_err, p->tc_wait);
    if (tmax) return cudaErrorInvalidValue;
    return launch_col_c2r(in, ncols, p->S, in_img, p->fy, p->col_logB_y, mid, out, row0, rows_out,
                          out_pitch, out_img, os, batch, st);
}

// the band-limited interpolator on the register-resident FFT (fixed-length
// kernels in use, W = S, M = 2W, all three lengths with a schedule)
static bool fourier_fast(ft_plan p) {
    return p->use_fast_x && p->fw.stw && p->fm.stw && fourier_fast_ok(p->W, p->fm.N, p->S);
}

static cudaError_t nvmt_rows(ft_plan p, float2* ws, int batch, cudaStream_t st) {
    if (p->interp == FT_INTERP_FOURIER) {
        const size_t nu = (size_t)p->L * (p->W + 1), nx = (size_t)p->L * p->S;
        if (fourier_fast(p))
            return launch_nvmt_rows_fourier_fast(false, ws, p->W, p->S, p->Hp, p->L, p->fw, p->fm, p->fx, p->d_chirp,
                                                 p->d_chirp + nu, p->d_chirp + nu + nx, batch, st);
        return launch_nvmt_rows_fourier(ws, p->W, p->S, p->Hp, p->L, p->fw, p->fm, p->fx, p->d_chirp,
                                        p->d_chirp + nu, p->d_chirp + nu + nx, batch, st);
    }
    if (p->precision != FT_PRECISION_FP32 && p->S == 4096)
        return launch_nvmt_rows_tc4096(ws, p->W, p->Hp, p->L, p->interp, p->precision, p->d_tc_err, p->tc_wait,
                                       batch, st);
    if (p->use_fast_x)
        return launch_nvmt_rows_fast(ws, p->W, p->Hp, p->L, p->interp, p->fx, batch, st, p->pdl, p->d_tc_err,
                                     p->tc_wait);
    return launch_nvmt_rows(ws, p->W, p->S, p->Hp, p->L, p->interp, p->fx, p->row_logB_x, batch, st);
}

static cudaError_t nvmt_rows_adj(ft_plan p, float2* ws, int batch, cudaStream_t st) {
    if (p->interp == FT_INTERP_FOURIER) {
        const size_t nu = (size_t)p->L * (p->W + 1), nx = (size_t)p->L * p->S;
        if (fourier_fast(p))
            return launch_nvmt_rows_fourier_fast(true, ws, p->W, p->S, p->Hp, p->L, p->fw, p->fm, p->fx, p->d_chirp,
                                                 p->d_chirp + nu, p->d_chirp + nu + nx, batch, st);
        return launch_nvmt_rows_fourier_adj(ws, p->W, p->S, p->Hp, p->L, p->fw, p->fm, p->fx, p->d_chirp,
                                            p->d_chirp + nu, p->d_chirp + nu + nx, batch, st);
    }
    if (p->use_fast_x) return launch_nvmt_rows_adjoint_fast(ws, p->W, p->Hp, p->L, p->interp, p->fx, batch, st);
    return launch_nvmt_rows_adjoint(ws, p->W, p->S, p->Hp, p->L, p->interp, p->fx, p->row_logB_x, batch, st);
}

extern "C" {

const char* ft_status_string(ft_status s) {
    switch (s) {
        case FT_OK: return "ok";
        case FT_ERR_INVALID_ARG: return "invalid argument";
        case FT_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case FT_ERR_OOM: return "out of memory";
        case FT_ERR_CUDA: return "CUDA error";
        case FT_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* ft_last_error(void) { return g_last_error; }

int ft_debug_build(void) {
#ifdef FT_DEBUG
    return 1;
#else
    return 0;
#endif
}

ft_status ft_debug_flags(uint32_t* flags) {
    if (!flags) return FT_ERR_INVALID_ARG;
    *flags = 0;
    FT_CUDA(cudaDeviceSynchronize(), "ft_debug_flags");
    *flags = ft_debug_read_fast() | ft_debug_read_peak_sparse();
    return FT_OK;
}

ft_status ft_plan_create(ft_plan* out, int H, int W, int n_slope, int n_intercept, int interp) {
    return ft_plan_create_space(out, H, W, n_slope, n_intercept, interp, FT_SPACE_REGULAR);
}

ft_status ft_plan_create_space(ft_plan* out, int img_H, int img_W, int n_slope, int n_intercept, int interp,
                               int space) {
    if (!out) return FT_ERR_INVALID_ARG;
    *out = nullptr;
    if (interp != FT_INTERP_LINEAR && interp != FT_INTERP_CUBIC && interp != FT_INTERP_FOURIER)
        return FT_ERR_INVALID_ARG;
    if (space != FT_SPACE_REGULAR && space != FT_SPACE_INVERSE) return FT_ERR_INVALID_ARG;
    // the inverse space is the regular transform of the transposed image
    const int H = space == FT_SPACE_INVERSE ? img_W : img_H;
    const int W = space == FT_SPACE_INVERSE ? img_H : img_W;
    if (H < 1 || W < 2 || (W & 1) || n_slope < W || n_intercept < H) return FT_ERR_UNSUPPORTED_SIZE;
    FftLen fy = {}, fx = {}, fw = {}, fm = {};
    if (!factorize(n_intercept, &fy) || !factorize(n_slope, &fx)) return FT_ERR_UNSUPPORTED_SIZE;
    if (interp == FT_INTERP_FOURIER) {
        int M = W + n_slope;
        while (M <= FT_MAX_LENGTH && !factorize(M, &fm)) ++M;
        if (M > FT_MAX_LENGTH || !factorize(W, &fw)) return FT_ERR_UNSUPPORTED_SIZE;
    }

    ft_plan p = new (std::nothrow) ft_plan_s();
    if (!p) return FT_ERR_OOM;
    p->H = H;
    p->W = W;
    p->space = space;
    p->img_H = img_H;
    p->img_W = img_W;
    p->S = n_slope;
    p->Hp = n_intercept;
    p->L = n_intercept / 2 + 1;
    p->interp = interp;
    p->top = (n_intercept - H) / 2;
    p->tc_wait = FT_WAIT_CYCLES;
    p->fy = fy;
    p->fx = fx;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    const char* force = getenv("FT_FORCE_GENERIC");
    const bool generic = force && force[0] == '1';
    const bool fast_y = fs_has(fy.N), fast_x = fs_has(fx.N);
    // the column length's table is full, the row lengths' tables are seed tables
    const size_t sy = fast_y ? fs_twsize(fy.N, false) : 0, sx = fast_x ? fs_twsize(fx.N, true) : 0;
    // per-pass tables of the band-limited interpolator's lengths W and M
    const bool fast_w = fw.N && fs_has(fw.N), fast_m = fm.N && fs_has(fm.N);
    const size_t sw = fast_w ? fs_twsize(fw.N, true) : 0, smm = fast_m ? fs_twsize(fm.N, true) : 0;
    std::vector<float2> tw((size_t)fy.N + fx.N + sy + sx + fw.N + fm.N + sw + smm);
    twiddles(fy.N, tw.data());
    twiddles(fx.N, tw.data() + fy.N);
    if (fast_y) stage_twiddles(fy.N, tw.data(), tw.data() + fy.N + fx.N, false);
    if (fast_x) stage_twiddles(fx.N, tw.data() + fy.N, tw.data() + fy.N + fx.N + sy, true);
    const size_t wo = (size_t)fy.N + fx.N + sy + sx;
    if (fw.N) twiddles(fw.N, tw.data() + wo);
    if (fm.N) twiddles(fm.N, tw.data() + wo + fw.N);
    const size_t so = wo + fw.N + fm.N;
    if (fast_w) stage_twiddles(fw.N, tw.data() + wo, tw.data() + so, true);
    if (fast_m) stage_twiddles(fm.N, tw.data() + wo + fw.N, tw.data() + so + sw, true);
    e = cudaMalloc(&p->d_tw, tw.size() * sizeof(float2));
    if (e != cudaSuccess) {
        delete p;
        cuda_fail(e, "cudaMalloc(twiddles)");
        return FT_ERR_OOM;
    }
    e = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_tw);
        delete p;
        return cuda_fail(e, "cudaMemcpy(twiddles)");
    }
    // the error word of the device-side waits (bulk copies, tensor cores)
    e = cudaMalloc(&p->d_tc_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(p->d_tc_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        if (p->d_tc_err) cudaFree(p->d_tc_err);
        cudaFree(p->d_tw);
        delete p;
        return cuda_fail(e, "cudaMalloc(error word)");
    }
    p->fy.tw = p->d_tw;
    p->fx.tw = p->d_tw + fy.N;
    p->fy.stw = fast_y ? p->d_tw + fy.N + fx.N : nullptr;
    p->fx.stw = fast_x ? p->d_tw + fy.N + fx.N + sy : nullptr;
    if (interp == FT_INTERP_FOURIER) {
        p->fw = fw;
        p->fm = fm;
        p->fw.tw = p->d_tw + wo;
        p->fm.tw = p->d_tw + wo + fw.N;
        p->fw.stw = fast_w ? p->d_tw + so : nullptr;
        p->fm.stw = fast_m ? p->d_tw + so + sw : nullptr;
        const ft_status cs = build_chirps(p);
        if (cs != FT_OK) {
            ft_plan_destroy(p);
            return cs;
        }
    }
    // transforms per block: 2 ping-pong buffers of N x B complex within 96 KB
    const int cap = 96 * 1024 / (int)(2 * sizeof(float2));
    p->col_logB_y = log2_floor(cap / fy.N > 0 ? cap / fy.N : 1);
    if (p->col_logB_y > 4) p->col_logB_y = 4;
    const int rcap = 96 * 1024 / (int)sizeof(float2) / (W + 2 * n_slope);
    p->row_logB_x = log2_floor(rcap > 0 ? rcap : 1);
    if (p->row_logB_x > 4) p->row_logB_x = 4;
    p->col_logB_max = p->col_logB_y;
    p->row_logB_max = p->row_logB_x;
    p->use_fast_y = fast_y && !generic;
    p->use_fast_x = fast_x && !generic;
    p->variant = generic ? 1 : 0;
    const char* lanes = getenv("FT_LANES");
    p->lanes = lanes && atoi(lanes) > 1 ? FT_LANES : 1;
    // programmatic dependent launch of the fixed-length kernels that follow
    // another kernel (steps 2-3, step 4, the peak pass); FT_PDL=0 turns it off
    const char* pdl = getenv("FT_PDL");
    p->pdl = !(pdl && !strcmp(pdl, "0"));
    const char* pm = getenv("FT_PEAKS");
    p->peak_mode = pm && !strcmp(pm, "sparse") ? 1 : (pm && !strcmp(pm, "dense") ? 2 : 0);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || p->num_sms < 1)
        p->num_sms = 1;
    *out = p;
    return FT_OK;
}

ft_status ft_plan_destroy(ft_plan p) {
    if (!p) return FT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_ws(p);
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->d_chirp) cudaFree(p->d_chirp);
    if (p->d_tc_err) cudaFree(p->d_tc_err);
    if (p->d_img_host) cudaFree(p->d_img_host);
    if (p->d_map_host) cudaFree(p->d_map_host);
    if (p->d_peaks_host) cudaFree(p->d_peaks_host);
    for (cudaEvent_t e : p->prof_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : p->chunk_events) cudaEventDestroy(e);
    if (p->lane_fork) cudaEventDestroy(p->lane_fork);
    for (int j = 0; j < FT_LANES; ++j) {
        if (p->lane_streams[j]) cudaStreamDestroy(p->lane_streams[j]);
        if (p->lane_join[j]) cudaEventDestroy(p->lane_join[j]);
    }
    if (p->start_event) cudaEventDestroy(p->start_event);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    cudaSetDevice(cur);
    delete p;
    return FT_OK;
}

int ft_plan_variant_count(ft_plan p) { return p ? 5 : 0; }

ft_status ft_plan_set_variant(ft_plan p, int variant) {
    if (!p || variant < 0 || variant > 4) return FT_ERR_INVALID_ARG;
    const bool fy = p->fy.stw != nullptr, fx = p->fx.stw != nullptr;
    if (variant == 0) {
        p->use_fast_y = fy;
        p->use_fast_x = fx;
        p->col_logB_y = p->col_logB_max;
        p->row_logB_x = p->row_logB_max;
    } else {
        const int v = variant - 1;              // generic kernels, 1 or 2x fewer transforms per block
        p->use_fast_y = 0;
        p->use_fast_x = 0;
        p->col_logB_y = p->col_logB_max - ((v & 1) && p->col_logB_max > 0 ? 1 : 0);
        p->row_logB_x = p->row_logB_max - ((v & 2) && p->row_logB_max > 0 ? 1 : 0);
    }
    p->variant = variant;
    return FT_OK;
}

int ft_plan_get_variant(ft_plan p) { return p ? p->variant : -1; }

ft_status ft_plan_set_precision(ft_plan p, int precision) {
    if (!p || precision < FT_PRECISION_FP32 || precision > FT_PRECISION_BF16X6) return FT_ERR_INVALID_ARG;
    if (precision != FT_PRECISION_FP32) {
        if (!((p->S == 4096 && p->interp != FT_INTERP_FOURIER) || p->Hp == 4096))
            return ft_record_error(FT_ERR_UNSUPPORTED_SIZE,
                                   "split precision: a length-4096 transform (n_slope 4096 with the linear or "
                                   "cubic interpolator, or n_intercept 4096) is needed");
        int cur = 0;
        FT_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
        FT_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
        const cudaError_t e = tc_prepare();
        cudaSetDevice(cur);
        if (e != cudaSuccess) return ft_record_cuda(e, "tensor-core tables");
    }
    p->precision = precision;
    return FT_OK;
}

int ft_plan_get_precision(ft_plan p) { return p ? p->precision : -1; }

ft_status ft_plan_tc_errors(ft_plan p, uint32_t* flags) {
    if (!p || !flags) return FT_ERR_INVALID_ARG;
    *flags = 0;
    if (!p->d_tc_err) return FT_OK;
    int cur = 0;
    FT_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    FT_CUDA(cudaSetDevice(p->device), "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(flags, p->d_tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_tc_err, 0, sizeof(unsigned));
    cudaSetDevice(cur);
    FT_CUDA(e, "ft_plan_tc_errors");
    if (*flags & 1u)
        return ft_record_error(FT_ERR_TIMEOUT, "ft_plan_tc_errors: a wait for the tensor cores timed out; the rows "
                                               "of the blocks that gave up are incomplete");
    if (*flags & 2u)
        return ft_record_error(FT_ERR_TIMEOUT, "ft_plan_tc_errors: a wait for a bulk copy of the NVMT rows timed "
                                               "out; the rows of the blocks that gave up were not written");
    if (*flags & 4u)
        return ft_record_error(FT_ERR_TIMEOUT, "ft_plan_tc_errors: a wait for a tensor copy of step 4's columns "
                                               "timed out; the columns of the blocks that gave up were not written");
    if (*flags & 8u)
        return ft_record_error(FT_ERR_TIMEOUT, "ft_plan_tc_errors: a wait for a tensor copy of step 1's image "
                                               "columns timed out; the columns of the blocks that gave up were not "
                                               "written");
    return FT_OK;
}

ft_status ft_plan_set_wait_cycles(ft_plan p, int64_t cycles) {
    if (!p || cycles < 0) return FT_ERR_INVALID_ARG;
    p->tc_wait = cycles;
    return FT_OK;
}

int64_t ft_plan_get_wait_cycles(ft_plan p) { return p ? (int64_t)p->tc_wait : -1; }

ft_status ft_plan_inject_alloc_failures(ft_plan p, int count) {
    if (!p || count < 0) return FT_ERR_INVALID_ARG;
    p->alloc_failures = count;
    return FT_OK;
}

size_t ft_workspace_bytes(ft_plan p, int batch) {
    if (!p || batch <= 0) return 0;
    return aux_off(p, batch);
}


// Lanes: a batch of at least 2 FT_LANES images is split into FT_LANES contiguous
// parts run on plan-owned streams forked from and joined back into the caller's
// stream, so that one part's compute-bound kernels share the SMs with another
// part's memory-bound ones.  The parts use disjoint slices of the workspace and
// the same kernels, so results do not depend on the split.  Off by default
// (every kernel then runs alone on the caller's stream, one launch per step
// over the whole batch); FT_LANES=2 in the environment at plan creation turns
// it on.

static ft_status lanes_fork(ft_plan p, cudaStream_t st) {
    if (!p->lane_fork) {
        FT_CUDA(cudaEventCreateWithFlags(&p->lane_fork, cudaEventDisableTiming), "lane event");
        for (int j = 0; j < FT_LANES; ++j) {
            FT_CUDA(cudaStreamCreateWithFlags(&p->lane_streams[j], cudaStreamNonBlocking), "lane stream");
            FT_CUDA(cudaEventCreateWithFlags(&p->lane_join[j], cudaEventDisableTiming), "lane event");
        }
    }
    FT_CUDA(cudaEventRecord(p->lane_fork, st), "lane fork");
    for (int j = 0; j < FT_LANES; ++j) FT_CUDA(cudaStreamWaitEvent(p->lane_streams[j], p->lane_fork, 0), "lane wait");
    return FT_OK;
}

static ft_status lanes_join(ft_plan p, cudaStream_t st) {
    for (int j = 0; j < FT_LANES; ++j) {
        FT_CUDA(cudaEventRecord(p->lane_join[j], p->lane_streams[j]), "lane join");
        FT_CUDA(cudaStreamWaitEvent(st, p->lane_join[j], 0), "lane join wait");
    }
    return FT_OK;
}

static int use_lanes(ft_plan p, int batch) { return p->lanes > 1 && batch >= 2 * FT_LANES; }

int ft_forward_launches(ft_plan p, int batch) {
    if (!p || batch <= 0) return 0;
    return (p->space == FT_SPACE_INVERSE ? 1 : 0) + 3 * (use_lanes(p, batch) ? FT_LANES : 1);
}
int ft_peaks_launches(ft_plan p, int batch) {
    if (!p || batch <= 0) return 0;
    return 2 * (use_lanes(p, batch) ? FT_LANES : 1);
}

// split precision: the length-4096 column transforms on the tensor cores too
static bool tc_columns(ft_plan p);

// The tile shape of ft_detect's peak pass (the tiles whose maxima step 4
// writes), or false when ft_detect runs ft_forward and ft_peaks instead: step 4
// must be the fixed-length FP32 kernel on the caller's stream, and the pass's
// shared memory must fit.
// Whether the pass from tile maxima beats the per-tile key kernels for this
// call.  It runs one block per image, so it costs one image's serial chain per
// wave of images: selecting among the tiles, then batches of 32 tiles (one at
// 1024^2 and 2048^2 with top_k = 32, over 20 at 4096^2 with top_k = 100: the
// batch count grows like (tiles x top_k)^2), plus, for ft_peaks, one streaming
// read for the tile maxima.  The key kernels spread every cell over the whole GPU
// but have a fixed latency of two dependent kernels, the second also one block
// per image.  Constants in microseconds, fitted to GB300 measurements of
// ft_detect both ways (1024^2 with 1-128 images, 512^2, 2048^2 and 4096^2; the
// model picks the faster pass in all 15 cases).  The pass from tile maxima
// occupies only one multiprocessor per image, so plans whose calls share the GPU
// with others (ft_batch) always take it.  FT_PEAKS=sparse / dense at plan
// creation fixes the choice.
static bool sparse_is_faster(ft_plan p, int batch, int top_k, bool with_tile_max) {
    if (p->peak_mode) return p->peak_mode == 1;
    const double cells = (double)p->Hp * p->S, tiles = cells / 256.0;
    const int waves = (batch + p->num_sms - 1) / p->num_sms;
    const double x = tiles * top_k / 1.5e6;
    const double sparse = waves * (1.2e-3 * tiles + 12.0 * (1.0 + x * x)) + (with_tile_max ? 0.7e-6 * cells * batch : 0.0);
    const double dense = 1.6e-6 * cells * batch + 27.0;
    return sparse < dense;
}

static bool sparse_peaks(ft_plan p, int batch, int top_k, int* rows, int* cols, int* bands) {
    if (!p->use_fast_y || tc_columns(p) || use_lanes(p, batch)) return false;
    if (!c2r_tile_shape(p->Hp, rows, cols, bands)) return false;
    return peak_sparse_fits(*rows, *cols, top_k) && sparse_is_faster(p, batch, top_k, false);
}

// ft_peaks takes the pass from tile maxima (tiles of tile_max_shape)
static bool peaks_use_tile_max(ft_plan p, int batch, int top_k) {
    int tr, tc;
    tile_max_shape(&tr, &tc);
    return peak_sparse_fits(tr, tc, top_k) && sparse_is_faster(p, batch, top_k, true);
}

// scratch of ft_peaks: tile maxima, or the per-tile keys where the pass from
// tile maxima does not fit
static size_t tile_max_bytes(ft_plan p, int batch) {
    int tr, tc;
    tile_max_shape(&tr, &tc);
    return (size_t)batch * ((p->Hp + tr - 1) / tr) * ((p->S + tc - 1) / tc) * sizeof(unsigned);
}
static size_t peaks_scratch_bytes(ft_plan p, int batch, int top_k) {
    return peaks_use_tile_max(p, batch, top_k) ? tile_max_bytes(p, batch) : peaks_key_bytes(p->Hp, p->S, batch, top_k);
}

// bytes of ft_detect's tile maxima for this batch (0 when it runs ft_peaks)
static size_t tmax_bytes(ft_plan p, int batch, int top_k) {
    int rows, cols, bands;
    if (!sparse_peaks(p, batch, top_k, &rows, &cols, &bands)) return 0;
    return (size_t)batch * bands * ((p->S + cols - 1) / cols) * sizeof(unsigned);
}

int ft_detect_launches(ft_plan p, int batch, int top_k) {
    if (!p || batch <= 0 || top_k < 1 || top_k > FT_MAX_TOPK) return 0;
    int rows, cols, bands;
    if (sparse_peaks(p, batch, top_k, &rows, &cols, &bands)) return (p->space == FT_SPACE_INVERSE ? 1 : 0) + 4;
    return ft_forward_launches(p, batch) + ft_peaks_launches(p, batch);
}

// split precision: the length-4096 column transforms on the tensor cores too,
// through a column-major copy (cm) so that their column pairs are contiguous rows
static bool tc_columns(ft_plan p) { return p->precision != FT_PRECISION_FP32 && p->Hp == 4096; }
static size_t cm_elems(ft_plan p) {
    const size_t a = (size_t)p->H * p->W, b = (size_t)p->Hp * p->S;
    return a > b ? a : b;
}

static cudaError_t tc_r2c(ft_plan p, const float* src, float2* ws, float* cm, int nb, cudaStream_t st) {
    cudaError_t e = launch_transpose(src, cm, p->H, p->W, nb, st);
    if (e != cudaSuccess) return e;
    return launch_col_r2c_tc4096(cm, p->H, p->W, p->top, ws, p->L, p->S, p->precision, p->d_tc_err, p->tc_wait, nb,
                                 st);
}

static cudaError_t tc_c2r(ft_plan p, const float2* ws, float* d_map, float* cm, int nb, cudaStream_t st) {
    cudaError_t e = launch_col_c2r_tc4096(ws, p->L, p->S, cm, p->precision, p->d_tc_err, p->tc_wait, nb, st);
    if (e != cudaSuccess) return e;
    return launch_transpose(cm, d_map, p->S, p->Hp, nb, st);
}

// Steps 1-4 of nb images; tmax (fixed-length FP32 step 4 only, else NULL) gets
// the tile maxima of |map| for the peak pass of ft_detect; follows_peak: step 1
// comes right after the peak pass of the previous batch of ft_detect_batches.
static ft_status forward_part(ft_plan p, const float* src, float* d_map, float2* ws, float* cm, int nb,
                              cudaStream_t st, unsigned* tmax = nullptr, bool follows_peak = false) {
    const bool tc_cols = tc_columns(p);
    FT_LAUNCH(p, FT_KERNEL_COL_R2C, st,
              tc_cols ? tc_r2c(p, src, ws, cm, nb, st)
                      : col_r2c(p, src, p->H, p->W, p->W, (size_t)p->H * p->W, p->top, ws, 1.f, 1.f, nb, st,
                                follows_peak),
              "step 1 (column R2C)");
    FT_LAUNCH(p, FT_KERNEL_NVMT_ROWS, st, nvmt_rows(p, ws, nb, st), "steps 2-3 (NVMT + row FFT)");
    FT_LAUNCH(p, FT_KERNEL_COL_C2R, st,
              tc_cols ? tc_c2r(p, ws, d_map, cm, nb, st)
                      : col_c2r(p, ws, p->S, 1.f, d_map, 0, p->Hp, p->S, (size_t)p->Hp * p->S, 1.f / (float)p->Hp,
                                nb, st, tmax),
              "step 4 (column C2R)");
    return FT_OK;
}

ft_status ft_forward(ft_plan p, const float* d_img, float* d_map, int batch, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_img || !d_map || ((uintptr_t)d_img & 7) || ((uintptr_t)d_map & 7)) return FT_ERR_INVALID_ARG;
    // the column-major copies of the split-precision path live in the aux region
    const size_t cm_bytes = tc_columns(p) ? (size_t)batch * cm_elems(p) * sizeof(float) : 0;
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, aux_off(p, batch) + cm_bytes, "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float2* ws = (float2*)p->d_ws;
    float* cm = (float*)((char*)p->d_ws + aux_off(p, batch));
    const float* src = d_img;
    if (p->space == FT_SPACE_INVERSE) {
        float* tp = (float*)((char*)p->d_ws + tposed_off(p, batch));
        FT_CUDA(launch_transpose(d_img, tp, p->img_H, p->img_W, batch, st), "transpose (inverse space)");
        src = tp;
    }
    if (!use_lanes(p, batch)) return forward_part(p, src, d_map, ws, cm, batch, st);
    if ((s = lanes_fork(p, st)) != FT_OK) return s;
    for (int j = 0; j < FT_LANES; ++j) {
        const int b0 = batch * j / FT_LANES, b1 = batch * (j + 1) / FT_LANES;
        s = forward_part(p, src + (size_t)b0 * p->H * p->W, d_map + (size_t)b0 * p->Hp * p->S,
                         ws + (size_t)b0 * p->L * p->S, cm + (size_t)b0 * cm_elems(p), b1 - b0, p->lane_streams[j]);
        if (s != FT_OK) return s;
    }
    return lanes_join(p, st);
}

// the adjoint after its first step (the spectrum of the map gradient is in ws)
static ft_status backward_tail(ft_plan p, float2* ws, float* d_grad_img, int batch, cudaStream_t st) {
    float* gdst = d_grad_img;
    if (p->space == FT_SPACE_INVERSE) gdst = (float*)((char*)p->d_ws + tposed_off(p, batch));
    FT_LAUNCH(p, FT_KERNEL_NVMT_ROWS_ADJ, st, nvmt_rows_adj(p, ws, batch, st), "adjoint of steps 2-3");
    FT_LAUNCH(p, FT_KERNEL_COL_C2R, st,
              col_c2r(p, ws, p->W, 0.5f, gdst, p->top, p->H, p->W, (size_t)p->H * p->W, 1.f, batch, st),
              "adjoint of step 1");
    if (p->space == FT_SPACE_INVERSE)
        FT_CUDA(launch_transpose(gdst, d_grad_img, p->H, p->W, batch, st), "transpose back (inverse space)");
    return FT_OK;
}

ft_status ft_backward(ft_plan p, const float* d_grad_map, float* d_grad_img, int batch, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_grad_map || !d_grad_img || ((uintptr_t)d_grad_map & 7) || ((uintptr_t)d_grad_img & 7))
        return FT_ERR_INVALID_ARG;
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, aux_off(p, batch), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float2* ws = (float2*)p->d_ws;
    const float inv = 1.f / (float)p->Hp;
    FT_LAUNCH(p, FT_KERNEL_COL_R2C, st,
              col_r2c(p, d_grad_map, p->Hp, p->S, p->S, (size_t)p->Hp * p->S, 0, ws, inv, 2.f * inv, batch, st),
              "adjoint of step 4");
    return backward_tail(p, ws, d_grad_img, batch, st);
}

ft_status ft_abs_mse_backward(ft_plan p, const float* d_map, const float* d_target, int batch, float scale,
                              float* d_loss, float* d_grad_img, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_map || !d_target || !d_loss || !d_grad_img || ((uintptr_t)d_map & 7) || ((uintptr_t)d_target & 7) ||
        ((uintptr_t)d_grad_img & 7))
        return FT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)p->Hp * p->S;
    const size_t off = aux_off(p, batch);
    if (!p->use_fast_y) {
        // no fused kernel for this length: the loss gradient through the workspace
        const size_t gbytes = (batch * cells * sizeof(float) + 255) & ~(size_t)255;
        ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + gbytes + loss_partial_bytes(batch),
                             "cudaMalloc(workspace)");
        if (s != FT_OK) return s;
        float* gmap = (float*)((char*)p->d_ws + off);
        FT_LAUNCH(p, FT_KERNEL_LOSS, st,
                  launch_abs_mse_grad(d_map, d_target, batch, cells, scale, d_loss, gmap,
                                      (float*)((char*)p->d_ws + off + gbytes), st),
                  "loss");
        return ft_backward(p, gmap, d_grad_img, batch, stream);
    }
    const int nblk = col_r2c_loss_blocks(p->fy, p->S);
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + (size_t)batch * nblk * sizeof(float), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    float2* ws = (float2*)p->d_ws;
    float* partial = (float*)((char*)p->d_ws + off);
    const float inv = 1.f / (float)p->Hp;
    const float gscale = (float)(1.0 / ((double)batch * (double)cells));
    FT_LAUNCH(p, FT_KERNEL_COL_R2C, st,
              launch_col_r2c_loss_fast(d_map, d_target, p->S, p->fy, ws, p->S, (size_t)p->L * p->S, inv, 2.f * inv,
                                       scale, gscale, partial, batch, st, p->d_tc_err, p->tc_wait),
              "loss and adjoint of step 4");
    FT_LAUNCH(p, FT_KERNEL_LOSS, st, launch_loss_finish(partial, nblk, cells, d_loss, batch, st), "loss");
    return backward_tail(p, ws, d_grad_img, batch, st);
}

ft_status ft_peaks(ft_plan p, const float* d_map, int batch, int top_k, float threshold,
                   ft_peak* d_out, int32_t* d_count, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (top_k < 1 || top_k > FT_MAX_TOPK || threshold != threshold) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_map || !d_out || !d_count) return FT_ERR_INVALID_ARG;
    // Tile maxima of the maps (one streaming read), then the peak pass that reads
    // only the tiles able to hold one of the top_k peaks; the per-tile key kernels
    // where that pass does not fit.  Scratch after the spectrum workspace.
    int tr, tc;
    tile_max_shape(&tr, &tc);
    const bool sparse = peaks_use_tile_max(p, batch, top_k);
    const size_t tpi = (size_t)((p->Hp + tr - 1) / tr) * ((p->S + tc - 1) / tc);     // tiles per map
    const size_t off = aux_off(p, batch);
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + peaks_scratch_bytes(p, batch, top_k), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    unsigned* tmax = (unsigned*)((char*)p->d_ws + off);
    unsigned long long* kbuf = (unsigned long long*)((char*)p->d_ws + off);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* bounds = peaks_bounds(kbuf, p->Hp, p->S, batch, top_k);
    const size_t kpi = peaks_tile_keys(p->Hp, p->S, top_k);
    const int lanes = use_lanes(p, batch) ? FT_LANES : 1;
    if (lanes > 1 && (s = lanes_fork(p, st)) != FT_OK) return s;
    for (int j = 0; j < lanes; ++j) {
        const int b0 = batch * j / lanes, b1 = batch * (j + 1) / lanes;
        cudaStream_t ls = lanes > 1 ? p->lane_streams[j] : st;
        const float* m = d_map + (size_t)b0 * p->Hp * p->S;
        if (sparse) {
            FT_LAUNCH(p, FT_KERNEL_TILE_MAX, ls,
                      launch_tile_max(m, p->Hp, p->S, b1 - b0, tmax + b0 * tpi, ls),
                      "peak detection (tile maxima)");
            FT_LAUNCH(p, FT_KERNEL_PEAK_SPARSE, ls,
                      launch_peak_sparse(m, tmax + b0 * tpi, p->Hp, p->S, tr, tc, b1 - b0, top_k, threshold,
                                         d_out + (size_t)b0 * top_k, d_count + b0, ls),
                      "peak detection (from tile maxima)");
            continue;
        }
        FT_LAUNCH(p, FT_KERNEL_PEAK_TILES, ls,
                  launch_peak_tiles(m, p->Hp, p->S, b1 - b0, top_k, threshold, kbuf + b0 * kpi, bounds + 2 * b0,
                                    ls),
                  "peak detection (tiles)");
        FT_LAUNCH(p, FT_KERNEL_PEAK_SELECT, ls,
                  launch_peak_select(kbuf + b0 * kpi, bounds + 2 * b0, p->Hp, p->S, b1 - b0, top_k,
                                     d_out + (size_t)b0 * top_k, d_count + b0, ls),
                  "peak detection (select)");
    }
    if (lanes > 1) return lanes_join(p, st);
    return FT_OK;
}

ft_status ft_detect(ft_plan p, const float* d_img, float* d_map, int batch, int top_k, float threshold,
                    ft_peak* d_out, int32_t* d_count, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (top_k < 1 || top_k > FT_MAX_TOPK || threshold != threshold) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_img || !d_map || !d_out || !d_count || ((uintptr_t)d_img & 7) || ((uintptr_t)d_map & 7))
        return FT_ERR_INVALID_ARG;
    int rows, cols, bands;
    if (!sparse_peaks(p, batch, top_k, &rows, &cols, &bands)) {
        const ft_status s = ft_forward(p, d_img, d_map, batch, stream);
        return s != FT_OK ? s : ft_peaks(p, d_map, batch, top_k, threshold, d_out, d_count, stream);
    }
    // the tile maxima [batch][bands][column blocks] live in the aux region
    const size_t off = aux_off(p, batch);
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + tmax_bytes(p, batch, top_k), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float2* ws = (float2*)p->d_ws;
    unsigned* tmax = (unsigned*)((char*)p->d_ws + off);
    const float* src = d_img;
    if (p->space == FT_SPACE_INVERSE) {
        float* tp = (float*)((char*)p->d_ws + tposed_off(p, batch));
        FT_CUDA(launch_transpose(d_img, tp, p->img_H, p->img_W, batch, st), "transpose (inverse space)");
        src = tp;
    }
    if ((s = forward_part(p, src, d_map, ws, nullptr, batch, st, tmax)) != FT_OK) return s;
    FT_LAUNCH(p, FT_KERNEL_PEAK_SPARSE, st,
              launch_peak_sparse(d_map, tmax, p->Hp, p->S, rows, cols, batch, top_k, threshold, d_out, d_count, st,
                                 p->pdl),
              "peak detection (tile maxima)");
    return FT_OK;
}

ft_status ft_detect_batches(ft_plan p, const float* const* d_imgs, int nb, int batch, float* d_map, int top_k,
                            float threshold, ft_peak* d_out, int32_t* d_count, void* stream) {
    if (!p || nb < 0 || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (top_k < 1 || top_k > FT_MAX_TOPK || threshold != threshold) return FT_ERR_INVALID_ARG;
    if (nb == 0 || batch == 0) return FT_OK;
    if (!d_imgs || !d_map || !d_out || !d_count || ((uintptr_t)d_map & 7)) return FT_ERR_INVALID_ARG;
    for (int j = 0; j < nb; ++j)
        if (!d_imgs[j] || ((uintptr_t)d_imgs[j] & 7)) return FT_ERR_INVALID_ARG;
    const size_t recs = (size_t)batch * top_k;
    int rows, cols, bands;
    // the pipeline needs step 1 on the fixed-length kernel right after the peak
    // pass from tile maxima; otherwise one ft_detect per batch
    const bool pipe = p->pdl && p->use_fast_y && !tc_columns(p) && p->space != FT_SPACE_INVERSE &&
                      sparse_peaks(p, batch, top_k, &rows, &cols, &bands);
    if (!pipe) {
        for (int j = 0; j < nb; ++j) {
            const ft_status s = ft_detect(p, d_imgs[j], d_map, batch, top_k, threshold, d_out + j * recs,
                                          d_count + (size_t)j * batch, stream);
            if (s != FT_OK) return s;
        }
        return FT_OK;
    }
    const size_t off = aux_off(p, batch);
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + tmax_bytes(p, batch, top_k), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float2* ws = (float2*)p->d_ws;
    unsigned* tmax = (unsigned*)((char*)p->d_ws + off);
    for (int j = 0; j < nb; ++j) {
        if ((s = forward_part(p, d_imgs[j], d_map, ws, nullptr, batch, st, tmax, j > 0)) != FT_OK) return s;
        FT_LAUNCH(p, FT_KERNEL_PEAK_SPARSE, st,
                  launch_peak_sparse(d_map, tmax, p->Hp, p->S, rows, cols, batch, top_k, threshold, d_out + j * recs,
                                     d_count + (size_t)j * batch, st, p->pdl),
                  "peak detection (tile maxima)");
    }
    return FT_OK;
}

ft_status ft_abs_mse_grad(ft_plan p, const float* d_map, const float* d_target, int batch, float scale,
                          float* d_loss, float* d_grad_map, void* stream) {
    if (!p || batch < 0 || batch > 65535) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_map || !d_target || !d_loss) return FT_ERR_INVALID_ARG;
    const size_t off = aux_off(p, batch);
    ft_status s = ensure(p, &p->d_ws, &p->ws_bytes, off + loss_partial_bytes(batch), "cudaMalloc(workspace)");
    if (s != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    FT_LAUNCH(p, FT_KERNEL_LOSS, st,
              launch_abs_mse_grad(d_map, d_target, batch, (size_t)p->Hp * p->S, scale, d_loss, d_grad_map,
                                  (float*)((char*)p->d_ws + off), st),
              "loss");
    return FT_OK;
}

ft_status ft_verify(ft_plan p, const float* d_img, const ft_peak* d_peaks, const int32_t* d_count, int batch,
                    int top_k, int half_width, float min_contrast, int32_t min_length, float* d_profile,
                    int32_t* d_length, int32_t* d_verdict, void* stream) {
    if (!p || batch < 0 || batch > 65535 || top_k < 1 || top_k > FT_MAX_TOPK) return FT_ERR_INVALID_ARG;
    if (half_width < 1 || half_width > 3) return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!d_img || !d_peaks || !d_count || !d_profile || !d_length || !d_verdict) return FT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // the transform's frame: the image itself, or its transpose in the inverse space
    const bool inv = p->space == FT_SPACE_INVERSE;
    const int stride_v = inv ? 1 : p->W, stride_u = inv ? p->img_W : 1;
    FT_LAUNCH(p, FT_KERNEL_VERIFY, st,
              launch_verify(d_img, p->H, p->W, stride_v, stride_u, (size_t)p->img_H * p->img_W, p->S, p->Hp, d_peaks,
                            d_count, batch, top_k, half_width, min_contrast, min_length, d_profile, d_length,
                            d_verdict, st),
              "line verification");
    return FT_OK;
}

ft_status ft_tc_dft64(const void* d_x, void* d_y, int nvec, int sign, int precision, uint32_t* d_err,
                      void* stream) {
    if (!d_x || !d_y || !d_err || nvec < 0 || (sign != 1 && sign != -1)) return FT_ERR_INVALID_ARG;
    if (precision != FT_PRECISION_BF16X3 && precision != FT_PRECISION_FP16X3) return FT_ERR_INVALID_ARG;
    if (nvec == 0) return FT_OK;
    FT_CUDA(launch_tc_dft64((const float2*)d_x, (float2*)d_y, nvec, sign, precision == FT_PRECISION_BF16X3 ? 1 : 0,
                            d_err, (cudaStream_t)stream),
            "ft_tc_dft64");
    return FT_OK;
}

ft_status ft_profile_enable(ft_plan p, int enable) {
    if (!p) return FT_ERR_INVALID_ARG;
    p->prof_on = enable ? 1 : 0;
    return FT_OK;
}

ft_status ft_profile_read(ft_plan p, double* total_ms, int32_t* launches, int n) {
    if (!p || n < 0 || (n > 0 && (!total_ms || !launches))) return FT_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        total_ms[i] = 0.0;
        launches[i] = 0;
    }
    ft_status st = FT_OK;
    for (size_t r = 0; r < p->prof_ids.size(); ++r) {
        cudaEvent_t a = p->prof_pool[2 * r], b = p->prof_pool[2 * r + 1];
        cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "ft_profile_read");
            break;
        }
        const int id = p->prof_ids[r];
        if (id < n) {
            total_ms[id] += ms;
            launches[id] += 1;
        }
    }
    p->prof_ids.clear();
    p->prof_used = 0;
    return st;
}

const char* ft_kernel_name(int id) {
    switch (id) {
        case FT_KERNEL_COL_R2C: return "k_col_r2c";
        case FT_KERNEL_NVMT_ROWS: return "k_nvmt_rows";
        case FT_KERNEL_COL_C2R: return "k_col_c2r";
        case FT_KERNEL_PEAK_TILES: return "k_peak_tiles";
        case FT_KERNEL_PEAK_SELECT: return "k_peak_select";
        case FT_KERNEL_NVMT_ROWS_ADJ: return "k_nvmt_rows_adjoint";
        case FT_KERNEL_LOSS: return "k_abs_mse_grad";
        case FT_KERNEL_VERIFY: return "k_verify";
        case FT_KERNEL_PEAK_SPARSE: return "k_peak_sparse";
        case FT_KERNEL_TILE_MAX: return "k_tile_max";
    }
    return "unknown";
}

ft_status ft_detect_host(ft_plan p, const float* h_img, int batch, int top_k, float threshold,
                         ft_peak* h_out, int32_t* h_count, void* stream) {
    if (!p || batch < 0 || batch > 65535 || top_k < 1 || top_k > FT_MAX_TOPK || threshold != threshold)
        return FT_ERR_INVALID_ARG;
    if (batch == 0) return FT_OK;
    if (!h_img || !h_out || !h_count) return FT_ERR_INVALID_ARG;
    const size_t img_px = (size_t)p->img_H * p->img_W;
    const size_t map_px = (size_t)p->Hp * p->S;
    const size_t img_b = (size_t)batch * img_px * sizeof(float);
    const size_t map_b = (size_t)batch * map_px * sizeof(float);
    const size_t pk_b = (size_t)batch * top_k * sizeof(ft_peak);
    const size_t cnt_off = (pk_b + 255) & ~(size_t)255;
    ft_status s;
    if ((s = ensure(p, (void**)&p->d_img_host, &p->img_host_bytes, img_b, "cudaMalloc(image)")) != FT_OK) return s;
    if ((s = ensure(p, (void**)&p->d_map_host, &p->map_host_bytes, map_b, "cudaMalloc(map)")) != FT_OK) return s;
    if ((s = ensure(p, (void**)&p->d_peaks_host, &p->peaks_host_bytes, cnt_off + batch * sizeof(int32_t),
                    "cudaMalloc(peaks)")) != FT_OK)
        return s;
    p->d_count_host = (int32_t*)((char*)p->d_peaks_host + cnt_off);
    // Chunks of images: the copy stream uploads chunk c + 1 while the caller's
    // stream transforms chunk c; peaks and counts come back per chunk.
    const int chunk = batch < FT_DETECT_CHUNK ? batch : FT_DETECT_CHUNK;
    const int nchunks = (batch + chunk - 1) / chunk;
    if (!p->copy_stream) FT_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
    if (!p->start_event) FT_CUDA(cudaEventCreateWithFlags(&p->start_event, cudaEventDisableTiming), "event");
    while ((int)p->chunk_events.size() < nchunks) {
        cudaEvent_t e;
        FT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        p->chunk_events.push_back(e);
    }
    // size the workspace for one chunk before any copy is in flight (the larger
    // of the two peak passes' scratch: tile maxima or per-tile keys)
    // (a smaller last chunk may take the other peak pass: room for every kind)
    size_t peak_b = tmax_bytes(p, chunk, top_k);
    if (tile_max_bytes(p, chunk) > peak_b) peak_b = tile_max_bytes(p, chunk);
    if (peaks_key_bytes(p->Hp, p->S, chunk, top_k) > peak_b) peak_b = peaks_key_bytes(p->Hp, p->S, chunk, top_k);
    const size_t need = aux_off(p, chunk) + peak_b;
    if ((s = ensure(p, &p->d_ws, &p->ws_bytes, need, "cudaMalloc(workspace)")) != FT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    FT_CUDA(cudaEventRecord(p->start_event, st), "event");
    FT_CUDA(cudaStreamWaitEvent(p->copy_stream, p->start_event, 0), "copy stream wait");
    for (int c = 0; c < nchunks; ++c) {
        const int b0 = c * chunk, nb = (batch - b0) < chunk ? (batch - b0) : chunk;
        FT_CUDA(cudaMemcpyAsync(p->d_img_host + b0 * img_px, h_img + b0 * img_px, nb * img_px * sizeof(float),
                                cudaMemcpyHostToDevice, p->copy_stream),
                "copy image in");
        FT_CUDA(cudaEventRecord(p->chunk_events[c], p->copy_stream), "event");
    }
    for (int c = 0; c < nchunks; ++c) {
        const int b0 = c * chunk, nb = (batch - b0) < chunk ? (batch - b0) : chunk;
        FT_CUDA(cudaStreamWaitEvent(st, p->chunk_events[c], 0), "wait for chunk");
        if ((s = ft_detect(p, p->d_img_host + b0 * img_px, p->d_map_host + b0 * map_px, nb, top_k, threshold,
                           p->d_peaks_host + (size_t)b0 * top_k, p->d_count_host + b0, stream)) != FT_OK)
            return s;
        FT_CUDA(cudaMemcpyAsync(h_out + (size_t)b0 * top_k, p->d_peaks_host + (size_t)b0 * top_k,
                                (size_t)nb * top_k * sizeof(ft_peak), cudaMemcpyDeviceToHost, st),
                "copy peaks out");
    }
    FT_CUDA(cudaMemcpyAsync(h_count, p->d_count_host, batch * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
            "copy counts out");
    FT_CUDA(cudaStreamSynchronize(st), "synchronise");
    return FT_OK;
}

}  // extern "C"
