// Mixed-size batches: many images of uneven sizes through the funnel transform
// and the peak detection in one graph launch, with a small autotuner.
//
// The batch fixes a packed layout: images (and maps, and peak rows) are stored
// back to back in the order of ft_batch_layout, which groups equal shapes
// together (largest first).  Every shape group has its own plan (tables and
// workspace), so the groups are independent and run on up to
// FT_BATCH_MAX_STREAMS side streams forked from and joined back into the
// caller's stream.  With FT_BATCH_GRAPH the whole fork / launches / join
// sequence is captured once into a CUDA graph (after an uncaptured run that
// allocates every workspace) and replayed while the arguments stay the same.
//
// The autotuner (FT_BATCH_TUNE) times every kernel variant of every group's
// plan (ft_plan_set_variant) on the caller's buffers and keeps the fastest; the
// choices are stored in a JSON file keyed by GPU name, shape and interpolator
// and reused by later batches.
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
    ft_plan plan;
    float tuned_ms;
};

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
};

static const char* interp_name(int i) { return i == FT_INTERP_LINEAR ? "linear" : "cubic"; }

static std::string cache_key(const ft_batch_s* b, const Group& g) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%dx%d|%s", b->gpu.c_str(), g.H, g.W, interp_name(b->interp));
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
    for (const Group& g : b->groups) {
        const std::string key = cache_key(b, g);
        char v[128];
        snprintf(v, sizeof(v), "{\"variant\": %d, \"ms\": %.6f}", ft_plan_get_variant(g.plan), g.tuned_ms);
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

// fork, per-group forward (+ peaks when top_k > 0), join
static ft_status enqueue(ft_batch_s* b, const float* imgs, float* maps, int top_k, float thr, ft_peak* out,
                         int32_t* cnt, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: fork");
    for (int s = 0; s < b->nstreams; ++s) {
        e = cudaStreamWaitEvent(b->streams[s], b->fork, 0);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: fork wait");
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group& g = b->groups[gi];
        cudaStream_t gs = b->streams[gi % b->nstreams];
        const float* img = imgs + b->img_off[g.start];
        float* gm = maps + b->map_off[g.start];
        const ft_status s = top_k > 0 ? ft_detect(g.plan, img, gm, g.count, top_k, thr, out + (size_t)g.start * top_k,
                                                  cnt + g.start, gs)
                                      : ft_forward(g.plan, img, gm, g.count, gs);
        if (s != FT_OK) return s;
    }
    for (int s = 0; s < b->nstreams; ++s) {
        e = cudaEventRecord(b->joins[s], b->streams[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->joins[s], 0);
        if (e != cudaSuccess) return ft_record_cuda(e, "ft_batch: join");
    }
    return FT_OK;
}

// time variant choices group by group on the caller's buffers; keep the fastest
static ft_status tune(ft_batch_s* b, const float* imgs, float* maps, int top_k, float thr, ft_peak* out,
                      int32_t* cnt, cudaStream_t st) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return ft_record_error(FT_ERR_CUDA, "ft_batch: event creation failed");
    ft_status rs = FT_OK;
    for (Group& g : b->groups) {
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
            Group g{H[i], W[i], j, 0, nullptr, 0.f};
            st = ft_plan_create(&g.plan, H[i], W[i], W[i], H[i], interp);
            if (st != FT_OK) break;
            // the groups run side by side: the peak pass that occupies one
            // multiprocessor per image (unless FT_PEAKS fixed it)
            if (g.plan->peak_mode == 0) g.plan->peak_mode = 1;
            const int v = cached.empty() ? -1 : cached_variant(cached, cache_key(b, g));
            if (v >= 0) ft_plan_set_variant(g.plan, v);
            b->groups.push_back(g);
        }
        b->groups.back().count += 1;
    }
    if (st == FT_OK) {
        b->nstreams = (int)std::min<size_t>(b->groups.size(), FT_BATCH_MAX_STREAMS);
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
    if (b->nstreams) cudaDeviceSynchronize();
    drop_graph(b);
    for (Group& g : b->groups) ft_plan_destroy(g.plan);
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
    info[4] = ft_plan_get_variant(gr.plan);
    return FT_OK;
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
