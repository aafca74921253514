// Mixed-size batches: many images of uneven sizes through the funnel transform
// and the peak detection, with a small autotuner.
//
// The batch fixes a packed layout: images (and maps, and peak rows) are stored
// back to back in the order of ft_batch_layout, which groups equal shapes
// together (largest first).  Images whose sides both have a fixed-length
// schedule up to 2048 (128, 192, 256, 384, 512, 768, 1024, 1536, 2048) with the
// linear or cubic interpolator run in the grouped kernels of k_batch.cu: one
// persistent launch per stage over all of them (step 1, steps 2-3, step 4 with
// tile maxima, the peak pass), fed by device work queues, with the batch's own
// workspace.  Every other shape group keeps a plan of its own (tables and
// workspace) and runs its ft_detect on one of up to FT_BATCH_MAX_STREAMS side
// streams forked from and joined back into the caller's stream.  With
// FT_BATCH_GRAPH the whole sequence is captured once into a CUDA graph (after an
// uncaptured run that allocates every workspace) and replayed while the
// arguments stay the same.
//
// The autotuner (FT_BATCH_TUNE) times every combination of the grouped kernels'
// threads per block (step 1: 256 or 512, steps 2-3: 128 or 256, step 4: 256 or
// 512, which fix the transforms per block of every length and the tile shape of
// the peak pass) on the caller's buffers and keeps the fastest, and times every
// kernel variant of the other groups' plans (ft_plan_set_variant).  The choices
// are stored in a JSON file keyed by GPU name and shapes and reused by later
// batches.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "ft_internal.cuh"

#define FT_BATCH_MAX_STREAMS 8

namespace {

struct Group {
    int H, W;
    int start, count;      // packed positions
    ft_plan plan;          // tables (grouped groups) or the whole path (the others)
    float tuned_ms;
    bool grouped;          // runs in the grouped kernels
};

// threads-per-block options of the grouped kernels, per stage (step 1, steps
// 2-3, step 4); the defaults are the per-plan kernels' shapes at length 1024
const int kThreadOpts[3][2] = {{256, 512}, {128, 256}, {256, 512}};
const int kDefaultThreads[3] = {512, 128, 256};

}  // namespace

struct ft_batch_s {
    int n = 0, interp = 0;
    std::vector<int32_t> order;             // packed position -> caller index
    std::vector<int64_t> img_off, map_off;  // per packed position, in elements
    int64_t img_total = 0, map_total = 0;
    std::vector<Group> groups;
    int nstreams = 0;
    cudaStream_t streams[FT_BATCH_MAX_STREAMS] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t joins[FT_BATCH_MAX_STREAMS] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_img = nullptr;
    void *g_map = nullptr, *g_out = nullptr, *g_cnt = nullptr, *g_stream = nullptr;
    int g_k = 0;
    float g_thr = 0.f;
    std::string cache;
    std::string gpu;
    // grouped path
    int ng = 0;                             // images in the grouped kernels
    int maxH = 0, maxW = 0;
    std::vector<BatchImg> himgs;            // host copy of the descriptors
    BatchImg* d_imgs = nullptr;
    int2* d_items[3][2] = {};               // (image, block) items per stage and threads option
    int nitems[3][2] = {};
    unsigned* d_queue = nullptr;            // one counter per stage
    float2* d_ws = nullptr;                 // half spectra of the grouped images
    unsigned* d_tmax = nullptr;             // tile maxima of step 4
    int threads[3] = {kDefaultThreads[0], kDefaultThreads[1], kDefaultThreads[2]};
    float tune_ms[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    int fallback_groups = 0;
};

static const char* interp_name(int i) { return i == FT_INTERP_LINEAR ? "linear" : "cubic"; }

static std::string cache_key(const ft_batch_s* b, const Group& g) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%dx%d|%s", b->gpu.c_str(), g.H, g.W, interp_name(b->interp));
    return buf;
}

// key of the grouped kernels' choice: GPU, interpolator and a digest (FNV-1a)
// of the grouped shapes with their counts
static std::string grouped_key(const ft_batch_s* b) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](unsigned v) {
        for (int k = 0; k < 4; ++k) {
            h ^= (v >> (8 * k)) & 255u;
            h *= 1099511628211ull;
        }
    };
    for (const Group& g : b->groups)
        if (g.grouped) {
            mix((unsigned)g.H);
            mix((unsigned)g.W);
            mix((unsigned)g.count);
        }
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|batch|%s|%016llx", b->gpu.c_str(), interp_name(b->interp), h);
    return buf;
}

static std::string read_file(const std::string& path) {
    std::string s;
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return s;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, k);
    fclose(f);
    return s;
}

// The cache is a flat JSON object {"key": {"variant": v, "ms": t}, ...}; this
// reader looks up one key's variant (-1 if absent or malformed).
static int cached_variant(const std::string& text, const std::string& key) {
    const std::string q = "\"" + key + "\"";
    size_t p = text.find(q);
    if (p == std::string::npos) return -1;
    p = text.find("\"variant\"", p + q.size());
    if (p == std::string::npos) return -1;
    p = text.find(':', p);
    if (p == std::string::npos) return -1;
    const int v = atoi(text.c_str() + p + 1);
    return (v >= 0 && v <= 4) ? v : -1;
}

// integer field `field` of the entry `key` (-1 if absent)
static int cached_field(const std::string& text, const std::string& key, const char* field) {
    const std::string q = "\"" + key + "\"";
    size_t p = text.find(q);
    if (p == std::string::npos) return -1;
    const size_t end = text.find('}', p);
    p = text.find(std::string("\"") + field + "\"", p + q.size());
    if (p == std::string::npos || p > end) return -1;
    p = text.find(':', p);
    if (p == std::string::npos) return -1;
    return atoi(text.c_str() + p + 1);
}

static void write_cache(const ft_batch_s* b) {
    if (b->cache.empty()) return;
    // keep the entries of other shapes / GPUs already in the file
    const std::string old = read_file(b->cache);
    std::vector<std::string> keys, vals;
    size_t p = 0;
    while ((p = old.find('"', p)) != std::string::npos) {
        const size_t e = old.find('"', p + 1);
        if (e == std::string::npos) break;
        const std::string key = old.substr(p + 1, e - p - 1);
        const size_t ob = old.find('{', e), cb = old.find('}', e);
        if (key.find('|') != std::string::npos && ob != std::string::npos && cb != std::string::npos && ob < cb) {
            keys.push_back(key);
            vals.push_back(old.substr(ob, cb - ob + 1));
            p = cb + 1;
        } else {
            p = e + 1;
        }
    }
    std::vector<std::pair<std::string, std::string>> entries;
    if (b->ng > 0) {
        float best = -1.f;
        for (float t : b->tune_ms)
            if (t > 0.f && (best < 0.f || t < best)) best = t;
        char v[160];
        snprintf(v, sizeof(v), "{\"r2c\": %d, \"rows\": %d, \"c2r\": %d, \"ms\": %.6f}", b->threads[0],
                 b->threads[1], b->threads[2], best);
        entries.emplace_back(grouped_key(b), v);
    }
    for (const Group& g : b->groups) {
        if (g.grouped) continue;
        char v[128];
        snprintf(v, sizeof(v), "{\"variant\": %d, \"ms\": %.6f}", ft_plan_get_variant(g.plan), g.tuned_ms);
        entries.emplace_back(cache_key(b, g), v);
    }
    for (const auto& en : entries) {
        const std::string& key = en.first;
        const char* v = en.second.c_str();
        auto it = std::find(keys.begin(), keys.end(), key);
        if (it == keys.end()) {
            keys.push_back(key);
            vals.push_back(v);
        } else {
            vals[it - keys.begin()] = v;
        }
    }
    const std::string tmp = b->cache + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < keys.size(); ++i)
        fprintf(f, "  \"%s\": %s%s\n", keys[i].c_str(), vals[i].c_str(), i + 1 < keys.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), b->cache.c_str());
}

static void drop_graph(ft_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

static int opt_index(int stage, int threads) { return threads == kThreadOpts[stage][1] ? 1 : 0; }

// the grouped kernels: queues cleared, then one launch per stage
static ft_status enqueue_grouped(ft_batch_s* b, const float* imgs, float* maps, int top_k, float thr, ft_peak* out,
                                 int32_t* cnt, cudaStream_t st) {
    if (b->ng == 0) return FT_OK;
    const int o0 = opt_index(0, b->threads[0]), o1 = opt_index(1, b->threads[1]), o2 = opt_index(2, b->threads[2]);
    cudaError_t e = cudaMemsetAsync(b->d_queue, 0, 4 * sizeof(unsigned), st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: clear the work queues");
    e = launch_batch_r2c(b->d_imgs, b->d_items[0][o0], b->nitems[0][o0], b->d_queue, imgs, b->d_ws, b->threads[0],
                         b->maxH, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: step 1 (grouped)");
    e = launch_batch_rows(b->d_imgs, b->d_items[1][o1], b->nitems[1][o1], b->d_queue + 1, b->d_ws, b->interp,
                          b->threads[1], b->maxW, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: steps 2-3 (grouped)");
    e = launch_batch_c2r(b->d_imgs, b->d_items[2][o2], b->nitems[2][o2], b->d_queue + 2, b->d_ws, maps,
                         top_k > 0 ? b->d_tmax : nullptr, b->threads[2], b->maxH, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: step 4 (grouped)");
    if (top_k > 0) {
        const size_t sm = batch_peaks_smem(b->himgs.data(), b->ng, b->threads[2], top_k);
        e = launch_batch_peaks(b->d_imgs, b->ng, b->d_queue + 3, maps, b->d_tmax, b->threads[2], top_k, thr, out, cnt,
                               sm, st);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: peaks (grouped)");
    }
    return FT_OK;
}

// fork, per-group forward (+ peaks when top_k > 0) of the groups outside the
// grouped kernels, the grouped kernels on the caller's stream, join
static ft_status enqueue(ft_batch_s* b, const float* imgs, float* maps, int top_k, float thr, ft_peak* out,
                         int32_t* cnt, cudaStream_t st) {
    cudaError_t e;
    if (b->nstreams > 0) {
        e = cudaEventRecord(b->fork, st);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: fork");
        for (int s = 0; s < b->nstreams; ++s) {
            e = cudaStreamWaitEvent(b->streams[s], b->fork, 0);
            if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: fork wait");
        }
    }
    int k = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group& g = b->groups[gi];
        if (g.grouped) continue;
        cudaStream_t gs = b->streams[k++ % b->nstreams];
        const float* img = imgs + b->img_off[g.start];
        float* gm = maps + b->map_off[g.start];
        const ft_status s = top_k > 0 ? ft_detect(g.plan, img, gm, g.count, top_k, thr, out + (size_t)g.start * top_k,
                                                  cnt + g.start, gs)
                                      : ft_forward(g.plan, img, gm, g.count, gs);
        if (s != FT_OK) return s;
    }
    const ft_status s = enqueue_grouped(b, imgs, maps, top_k, thr, out, cnt, st);
    if (s != FT_OK) return s;
    for (int j = 0; j < b->nstreams; ++j) {
        e = cudaEventRecord(b->joins[j], b->streams[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->joins[j], 0);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: join");
    }
    return FT_OK;
}

// Time the grouped kernels with every combination of threads per block (mean of
// 3 runs after one warm-up), and every plan variant of the other groups, group
// by group, on the caller's buffers; keep the fastest.
static ft_status tune(ft_batch_s* b, const float* imgs, float* maps, int top_k, float thr, ft_peak* out,
                      int32_t* cnt, cudaStream_t st) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ft_record_error(FT_ERR_CUDA, "ft_batch: event creation failed");
    ft_status rs = FT_OK;
    if (b->ng > 0) {
        float best_ms = 1e30f;
        int best = 0;
        for (int c = 0; c < 8 && rs == FT_OK; ++c) {
            for (int k = 0; k < 3; ++k) b->threads[k] = kThreadOpts[k][(c >> (2 - k)) & 1];
            for (int rep = 0; rep < 4 && rs == FT_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, st);
                rs = enqueue_grouped(b, imgs, maps, top_k, thr, out, cnt, st);
            }
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rs = ft_record_error(FT_ERR_CUDA, "ft_batch: tuning run failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            b->tune_ms[c] = ms / 3.f;
            if (b->tune_ms[c] < best_ms) {
                best_ms = b->tune_ms[c];
                best = c;
            }
        }
        for (int k = 0; k < 3; ++k) b->threads[k] = kThreadOpts[k][(best >> (2 - k)) & 1];
    }
    for (Group& g : b->groups) {
        if (g.grouped) continue;
        int best = 0;
        float best_ms = 1e30f;
        for (int v = 0; v < ft_plan_variant_count(g.plan) && rs == FT_OK; ++v) {
            if (ft_plan_set_variant(g.plan, v) != FT_OK) continue;
            const float* gi = imgs + b->img_off[g.start];
            float* gm = maps + b->map_off[g.start];
            for (int rep = 0; rep < 7 && rs == FT_OK; ++rep) {
                if (rep == 2) cudaEventRecord(e0, st);
                rs = top_k > 0 ? ft_detect(g.plan, gi, gm, g.count, top_k, thr, out + (size_t)g.start * top_k,
                                           cnt + g.start, st)
                               : ft_forward(g.plan, gi, gm, g.count, st);
            }
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rs = ft_record_error(FT_ERR_CUDA, "ft_batch: tuning run failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 5.f;
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        ft_plan_set_variant(g.plan, best);
        g.tuned_ms = best_ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs == FT_OK) write_cache(b);
    return rs;
}

// descriptors, work items and workspace of the grouped images
static ft_status setup_grouped(ft_batch_s* b) {
    std::vector<std::vector<int2>> items(6);
    long long ws = 0, tm = 0;
    for (const Group& g : b->groups) {
        if (!g.grouped) continue;
        int tiles = 0;
        for (int o = 0; o < 2; ++o) {
            int rows, cols, bands, nbx;
            batch_tile_shape(g.H, g.W, kThreadOpts[2][o], &rows, &cols, &bands, &nbx);
            if (bands * nbx > tiles) tiles = bands * nbx;
        }
        for (int j = g.start; j < g.start + g.count; ++j) {
            BatchImg d;
            d.img_off = b->img_off[j];
            d.map_off = b->map_off[j];
            d.ws_off = ws;
            d.tm_off = tm;
            d.H = g.H;
            d.W = g.W;
            d.pos = j;
            d.stw_y = g.plan->fy.stw;
            d.stw_x = g.plan->fx.stw;
            const int idx = (int)b->himgs.size();
            b->himgs.push_back(d);
            ws += (long long)(g.H / 2 + 1) * g.W;
            tm += tiles;
            for (int o = 0; o < 2; ++o) {
                for (int k = 0; k < batch_r2c_blocks(g.H, g.W, kThreadOpts[0][o]); ++k) items[0 + o].push_back(make_int2(idx, k));
                for (int k = 0; k < batch_rows_blocks(g.H, g.W, kThreadOpts[1][o]); ++k) items[2 + o].push_back(make_int2(idx, k));
                for (int k = 0; k < batch_c2r_blocks(g.H, g.W, kThreadOpts[2][o]); ++k) items[4 + o].push_back(make_int2(idx, k));
            }
        }
        if (g.H > b->maxH) b->maxH = g.H;
        if (g.W > b->maxW) b->maxW = g.W;
    }
    b->ng = (int)b->himgs.size();
    if (b->ng == 0) return FT_OK;
    cudaError_t e = cudaMalloc(&b->d_imgs, b->himgs.size() * sizeof(BatchImg));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_imgs, b->himgs.data(), b->himgs.size() * sizeof(BatchImg), cudaMemcpyHostToDevice);
    for (int st = 0; st < 3 && e == cudaSuccess; ++st)
        for (int o = 0; o < 2 && e == cudaSuccess; ++o) {
            const std::vector<int2>& v = items[2 * st + o];
            b->nitems[st][o] = (int)v.size();
            e = cudaMalloc(&b->d_items[st][o], v.size() * sizeof(int2));
            if (e == cudaSuccess) e = cudaMemcpy(b->d_items[st][o], v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice);
        }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ws, (size_t)ws * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tmax, (size_t)(tm > 0 ? tm : 1) * sizeof(unsigned));
    if (e != cudaSuccess) {
        ft_record_cuda(e, "ft_batch_create: grouped workspace");
        return e == cudaErrorMemoryAllocation ? FT_ERR_OOM : FT_ERR_CUDA;
    }
    return FT_OK;
}

extern "C" {

ft_status ft_batch_destroy(ft_batch b);

ft_status ft_batch_create(ft_batch* out, int n, const int32_t* H, const int32_t* W, int interp,
                          const char* tune_cache) {
    if (!out) return FT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !H || !W) return FT_ERR_INVALID_ARG;
    ft_batch b = new (std::nothrow) ft_batch_s();
    if (!b) return FT_ERR_OOM;
    b->n = n;
    b->interp = interp;
    if (tune_cache) b->cache = tune_cache;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) b->gpu = prop.name;
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
        const long long pa = (long long)H[a] * W[a], pc = (long long)H[c] * W[c];
        if (pa != pc) return pa > pc;
        if (H[a] != H[c]) return H[a] < H[c];
        return W[a] < W[c];
    });
    b->img_off.resize(n);
    b->map_off.resize(n);
    const std::string cached = b->cache.empty() ? std::string() : read_file(b->cache);
    ft_status st = FT_OK;
    for (int j = 0; j < n && st == FT_OK; ++j) {
        const int i = b->order[j];
        b->img_off[j] = b->img_total;
        b->map_off[j] = b->map_total;
        b->img_total += (int64_t)H[i] * W[i];
        b->map_total += (int64_t)H[i] * W[i];        // n_slope = W, n_intercept = H
        if (b->groups.empty() || b->groups.back().H != H[i] || b->groups.back().W != W[i]) {
            Group g{H[i], W[i], j, 0, nullptr, -1.f, false};
            st = ft_plan_create(&g.plan, H[i], W[i], W[i], H[i], interp);
            if (st != FT_OK) break;
            g.grouped = batch_len_ok(H[i]) && batch_len_ok(W[i]) && interp != FT_INTERP_FOURIER;
            // the other groups run side by side: the peak pass that occupies one
            // multiprocessor per image (unless FT_PEAKS fixed it)
            if (g.plan->peak_mode == 0) g.plan->peak_mode = 1;
            const int v = cached.empty() || g.grouped ? -1 : cached_variant(cached, cache_key(b, g));
            if (v >= 0) ft_plan_set_variant(g.plan, v);
            if (!g.grouped) b->fallback_groups += 1;
            b->groups.push_back(g);
        }
        b->groups.back().count += 1;
    }
    if (st == FT_OK) st = setup_grouped(b);
    if (st == FT_OK && b->ng > 0 && !cached.empty()) {
        const std::string key = grouped_key(b);
        const int t0 = cached_field(cached, key, "r2c"), t1 = cached_field(cached, key, "rows"),
                  t2 = cached_field(cached, key, "c2r");
        if (batch_threads_ok(0, t0) && batch_threads_ok(1, t1) && batch_threads_ok(2, t2)) {
            b->threads[0] = t0;
            b->threads[1] = t1;
            b->threads[2] = t2;
        }
    }
    if (st == FT_OK) {
        b->nstreams = std::min(b->fallback_groups, FT_BATCH_MAX_STREAMS);
        cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int s = 0; s < b->nstreams && e == cudaSuccess; ++s) {
            e = cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) st = ft_record_cuda(e, "ft_batch_create: streams");
    }
    if (st != FT_OK) {
        ft_batch_destroy(b);
        return st;
    }
    *out = b;
    return FT_OK;
}

ft_status ft_batch_destroy(ft_batch b) {
    if (!b) return FT_OK;
    if (b->nstreams || b->ng) cudaDeviceSynchronize();
    drop_graph(b);
    for (Group& g : b->groups) ft_plan_destroy(g.plan);
    if (b->d_imgs) cudaFree(b->d_imgs);
    for (int st = 0; st < 3; ++st)
        for (int o = 0; o < 2; ++o)
            if (b->d_items[st][o]) cudaFree(b->d_items[st][o]);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->d_ws) cudaFree(b->d_ws);
    if (b->d_tmax) cudaFree(b->d_tmax);
    for (int s = 0; s < FT_BATCH_MAX_STREAMS; ++s) {
        if (b->streams[s]) cudaStreamDestroy(b->streams[s]);
        if (b->joins[s]) cudaEventDestroy(b->joins[s]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return FT_OK;
}

ft_status ft_batch_layout(ft_batch b, int32_t* order, int64_t* img_off, int64_t* map_off, int64_t* totals) {
    if (!b) return FT_ERR_INVALID_ARG;
    for (int j = 0; j < b->n; ++j) {
        if (order) order[j] = b->order[j];
        if (img_off) img_off[j] = b->img_off[j];
        if (map_off) map_off[j] = b->map_off[j];
    }
    if (totals) {
        totals[0] = b->img_total;
        totals[1] = b->map_total;
    }
    return FT_OK;
}

int ft_batch_group_count(ft_batch b) { return b ? (int)b->groups.size() : 0; }

ft_status ft_batch_group_info(ft_batch b, int g, int32_t* info) {
    if (!b || g < 0 || g >= (int)b->groups.size() || !info) return FT_ERR_INVALID_ARG;
    const Group& gr = b->groups[g];
    info[0] = gr.H;
    info[1] = gr.W;
    info[2] = gr.start;
    info[3] = gr.count;
    info[4] = gr.grouped ? -1 : ft_plan_get_variant(gr.plan);
    return FT_OK;
}

ft_status ft_batch_config(ft_batch b, int32_t* info) {
    if (!b || !info) return FT_ERR_INVALID_ARG;
    info[0] = b->ng;
    info[1] = b->fallback_groups;
    info[2] = b->threads[0];
    info[3] = b->threads[1];
    info[4] = b->threads[2];
    info[5] = ft_batch_launches(b, 1);
    return FT_OK;
}

ft_status ft_batch_set_config(ft_batch b, int r2c_threads, int rows_threads, int c2r_threads) {
    if (!b || !batch_threads_ok(0, r2c_threads) || !batch_threads_ok(1, rows_threads) ||
        !batch_threads_ok(2, c2r_threads))
        return FT_ERR_INVALID_ARG;
    if (b->threads[0] != r2c_threads || b->threads[1] != rows_threads || b->threads[2] != c2r_threads) drop_graph(b);
    b->threads[0] = r2c_threads;
    b->threads[1] = rows_threads;
    b->threads[2] = c2r_threads;
    return FT_OK;
}

int ft_batch_tune_ms(ft_batch b, float* ms, int n) {
    if (!b) return 0;
    for (int i = 0; i < n && i < 8; ++i) ms[i] = b->tune_ms[i];
    return 8;
}

int ft_batch_launches(ft_batch b, int top_k) {
    if (!b || top_k < 0 || top_k > FT_MAX_TOPK) return 0;
    int n = b->ng > 0 ? (top_k > 0 ? 4 : 3) : 0;
    for (const Group& g : b->groups)
        if (!g.grouped)
            n += top_k > 0 ? ft_detect_launches(g.plan, g.count, top_k) : ft_forward_launches(g.plan, g.count);
    return n;
}

float ft_batch_group_tuned_ms(ft_batch b, int g) {
    return (b && g >= 0 && g < (int)b->groups.size()) ? b->groups[g].tuned_ms : -1.f;
}

ft_status ft_batch_run(ft_batch b, const float* d_imgs, float* d_maps, int top_k, float threshold,
                       ft_peak* d_out, int32_t* d_count, void* stream, int flags) {
    if (!b || !d_imgs || !d_maps) return FT_ERR_INVALID_ARG;
    if (top_k < 0 || top_k > FT_MAX_TOPK || (top_k > 0 && (!d_out || !d_count))) return FT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if ((flags & FT_BATCH_GRAPH) && !st) return FT_ERR_INVALID_ARG;   // the legacy stream cannot be captured
    ft_status s = FT_OK;
    if (flags & FT_BATCH_TUNE) {
        drop_graph(b);
        s = tune(b, d_imgs, d_maps, top_k, threshold, d_out, d_count, st);
        if (s != FT_OK) return s;
    }
    if (!(flags & FT_BATCH_GRAPH)) return enqueue(b, d_imgs, d_maps, top_k, threshold, d_out, d_count, st);
    const bool same = b->exec && b->g_img == d_imgs && b->g_map == d_maps && b->g_k == top_k &&
                      b->g_thr == threshold && b->g_out == d_out && b->g_cnt == d_count && b->g_stream == stream;
    if (!same) {
        drop_graph(b);
        // an uncaptured run first: it allocates every plan's workspace
        s = enqueue(b, d_imgs, d_maps, top_k, threshold, d_out, d_count, st);
        if (s != FT_OK) return s;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch_run: begin capture");
        s = enqueue(b, d_imgs, d_maps, top_k, threshold, d_out, d_count, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (s != FT_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch_run: end capture");
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return ft_record_cuda(e, "ft_batch_run: instantiate");
        }
        b->g_img = d_imgs;
        b->g_map = d_maps;
        b->g_k = top_k;
        b->g_thr = threshold;
        b->g_out = d_out;
        b->g_cnt = d_count;
        b->g_stream = stream;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch_run: graph launch");
    return FT_OK;
}

}  // extern "C"
