// Autotuner of the tiled forward kernel and its cache.
//
// The paper's question (Sec. IV, V) is whether one tile shape suits every
// GPU and every scale; its answer is that it does not always. Here every
// problem class (GPU, dtype, method, channel layout, coordinate mode, scale
// class per axis, output size class) gets its own tile shape, chosen by
// timing the candidates on the caller's buffers with CUDA events.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "capi_internal.h"

namespace rs {

struct Tuned {
    int tile_w, tile_h, threads;
};

static std::mutex g_tune_mu;
static std::map<std::string, Tuned> g_tune;
static bool g_env_loaded = false;

static int scale_class(int n, int m)
{
    return (int)std::lround(std::log2((double)m / (double)n) * 4.0);
}

static std::string tune_key(const Geom& g, int method, int dtype)
{
    const double elems = (double)g.Ho * g.Wo * g.C * g.planes;
    char buf[160];
    std::snprintf(buf, sizeof buf, "sms=%d;dt=%d;m=%d;C=%d;coord=%d;sy=%d;sx=%d;sz=%d", num_sms(), dtype,
                  method, g.C, g.coord, scale_class(g.H, g.Ho), scale_class(g.W, g.Wo),
                  (int)std::floor(std::log2(std::max(1.0, elems))));
    return buf;
}

static bool load_file(const char* path)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    std::map<std::string, Tuned> add;
    bool versioned = false;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, "# resample-tune v1", 18) == 0) { versioned = true; continue; }
        if (line[0] == '#' || line[0] == '\n') continue;
        char key[256];
        Tuned t;
        if (std::sscanf(line, "%255s %d %d %d", key, &t.tile_w, &t.tile_h, &t.threads) == 4 &&
            t.tile_w > 0 && t.tile_h > 0 && (t.threads == 128 || t.threads == 256))
            add[key] = t;
    }
    std::fclose(f);
    if (!versioned) return false;   // unknown or stale format: ignore the file
    for (auto& kv : add) g_tune[kv.first] = kv.second;
    return true;
}

static void load_env_once()
{
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char* p = std::getenv("RS_TUNE_CACHE");
    if (p && *p) load_file(p);
}

rs_status choose_tile(const Geom& g, int method, int dtype, const rs_options& o, TileCfg& cfg)
{
    if (o.tile_w || o.tile_h || o.threads) {
        TileCfg d = tiled_default(g, method);
        cfg = TileCfg{o.tile_w ? o.tile_w : d.tile_w, o.tile_h ? o.tile_h : d.tile_h,
                      o.threads ? o.threads : d.threads, 0, 0, 0};
        return tiled_config(g, method, cfg) ? RS_OK : RS_ERR_INVALID_ARG;
    }
    if (o.impl == RS_IMPL_AUTO) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_env_once();
        auto it = g_tune.find(tune_key(g, method, dtype));
        if (it != g_tune.end()) {
            cfg = TileCfg{it->second.tile_w, it->second.tile_h, it->second.threads, 0, 0, 0};
            if (tiled_config(g, method, cfg)) return RS_OK;
        }
    }
    cfg = tiled_default(g, method);
    return cfg.tile_w ? RS_OK : RS_ERR_UNSUPPORTED;
}

// Median time in microseconds of `reps` launches, measured as 3 batches.
static cudaError_t time_cfg(const Geom& g, int method, int dtype, const void* src, void* dst,
                            const TileCfg& cfg, cudaStream_t st, float* us)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
    float samples[3];
    int reps = 1;
    for (int k = -1; k < 3 && e == cudaSuccess; ++k) {
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_tiled(g, method, dtype, src, dst, cfg, st);
        cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (k < 0) {   // warm-up launch sizes the batches to ~2 ms each
            reps = std::max(1, std::min(50, (int)std::ceil(2.0f / std::max(ms, 1e-3f))));
        } else {
            samples[k] = 1000.0f * ms / reps;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    std::sort(samples, samples + 3);
    *us = samples[1];
    return cudaSuccess;
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_autotune(const void* src, const rs_layout* in, void* dst, const rs_layout* out,
                      rs_dtype dtype, rs_method method, const rs_options* opt, void* stream,
                      rs_tile_config* best)
{
    rs_options o = options_or_default(opt);
    Geom g;
    rs_status s = make_geom(src, in, dst, out, dtype, method, o, g);
    if (s != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    static const int widths[] = {128, 256, 512, 1024};
    static const int heights[] = {4, 8, 16, 32, 64};
    static const int threads[] = {128, 256};
    TileCfg def = tiled_default(g, method);
    if (!def.tile_w) return RS_ERR_UNSUPPORTED;
    float def_us = 0.0f;
    cudaError_t e = time_cfg(g, method, dtype, src, dst, def, st, &def_us);
    if (e != cudaSuccess) return cuda_status(e);
    TileCfg bestc = def;
    float best_us = def_us;
    int n = 1;
    for (int tw : widths)
        for (int th : heights)
            for (int nt : threads) {
                TileCfg c{tw, th, nt, 0, 0, 0};
                if (!tiled_config(g, method, c)) continue;
                if (c.tile_w == def.tile_w && c.tile_h == def.tile_h && c.threads == def.threads) continue;
                float us = 0.0f;
                e = time_cfg(g, method, dtype, src, dst, c, st, &us);
                if (e != cudaSuccess) return cuda_status(e);
                ++n;
                if (us < best_us) { best_us = us; bestc = c; }
            }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(g, method, dtype)] = Tuned{bestc.tile_w, bestc.tile_h, bestc.threads};
    }
    if (best) {
        best->tile_w = bestc.tile_w;
        best->tile_h = bestc.tile_h;
        best->threads = bestc.threads;
        best->best_us = best_us;
        best->default_us = def_us;
        best->candidates = n;
    }
    return RS_OK;
}

rs_status rs_tile_config_for(const rs_layout* in, const rs_layout* out, rs_dtype dtype, rs_method method,
                             const rs_options* opt, rs_tile_config* cfg)
{
    if (!cfg) return RS_ERR_INVALID_ARG;
    rs_options o = options_or_default(opt);
    Geom g;
    LayoutInfo li, lo;
    rs_status s = geom_from_layouts(in, out, dtype, method, o, g, li, lo);
    if (s != RS_OK) return s;
    TileCfg c;
    if ((s = choose_tile(g, method, dtype, o, c)) != RS_OK) return s;
    cfg->tile_w = c.tile_w;
    cfg->tile_h = c.tile_h;
    cfg->threads = c.threads;
    cfg->best_us = 0.0f;
    cfg->default_us = 0.0f;
    cfg->candidates = 0;
    return RS_OK;
}

rs_status rs_tune_cache_save(const char* path)
{
    if (!path) return RS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return RS_ERR_INVALID_ARG;
    std::fprintf(f, "# resample-tune v1\n");
    for (auto& kv : g_tune)
        std::fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.tile_w, kv.second.tile_h, kv.second.threads);
    std::fclose(f);
    return RS_OK;
}

rs_status rs_tune_cache_load(const char* path)
{
    if (!path) return RS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return load_file(path) ? RS_OK : RS_ERR_INVALID_ARG;
}

void rs_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // extern "C"
