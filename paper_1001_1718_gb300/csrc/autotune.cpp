// Kernel choice, autotuner and tuning cache of the forward path.
//
// The paper's question (Sec. IV, V) is whether one tile shape suits every
// GPU and every scale; its answer is that it does not always. Here every
// problem class (GPU model and CUDA runtime, SM count, dtype, method, channel
// layout, coordinate mode, scale class per axis, output size class) gets its
// own kernel and shape, chosen
// by timing the candidates on the caller's buffers with CUDA events.
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

static std::mutex g_tune_mu;
static std::map<std::string, Tuned> g_tune;
static bool g_env_loaded = false;
static void load_env_once();

static int scale_class(int n, int m)
{
    return (int)std::lround(std::log2((double)m / (double)n) * 4.0);
}

static std::string tune_key(const Geom& g, int method, int dtype)
{
    const double elems = (double)g.Ho * g.Wo * g.C * g.planes;
    char buf[160];
    std::snprintf(buf, sizeof buf, ";sms=%d;dt=%d;m=%d;C=%d;coord=%d;sy=%d;sx=%d;sz=%d", num_sms(), dtype,
                  method, g.C, g.coord, scale_class(g.H, g.Ho), scale_class(g.W, g.Wo),
                  (int)std::floor(std::log2(std::max(1.0, elems))));
    return "gpu=" + device_tag() + buf;
}

bool tune_lookup(const std::string& key, Tuned& t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_env_once();
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    t = it->second;
    return true;
}

void tune_store(const std::string& key, const Tuned& t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = t;
}

static bool valid_tuned(const Tuned& t)
{
    if (t.impl == RS_IMPL_GATHER) return t.tile_w > 0 && t.tile_h > 0;
    if (t.impl == RS_IMPL_WINDOW) return t.tile_h >= 0 && t.tile_w > 0 && (t.waves > 0 || t.tile_w <= 256);
    if (t.impl == RS_IMPL_STREAM) return t.tile_w > 0 && t.tile_h > 0 && t.waves > 0;
    if (t.impl == RS_IMPL_TILED) return t.tile_w > 0 && t.tile_h > 0 && (t.threads == 128 || t.threads == 256);
    if (t.impl == RS_IMPL_REDUCE) return true;
    return false;
}

static bool load_file(const char* path)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    std::map<std::string, Tuned> add;
    bool versioned = false;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, "# resample-tune v2", 18) == 0) { versioned = true; continue; }
        if (line[0] == '#' || line[0] == '\n') continue;
        char key[256];
        Tuned t;
        if (std::sscanf(line, "%255s %d %d %d %d %d", key, &t.impl, &t.tile_w, &t.tile_h, &t.threads, &t.waves) == 6 &&
            valid_tuned(t))
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

static bool make_choice(const Geom& g, int method, int dtype, const void* src, const Tuned& t, KernelChoice& k)
{
    k.impl = t.impl;
    if (t.impl == RS_IMPL_GATHER) {
        k.gather_w = t.tile_w;
        k.gather_rows = t.tile_h;
        return method == RS_NEAREST && nearest_config(g, dtype, t.tile_w, t.tile_h);
    }
    if (t.impl == RS_IMPL_WINDOW) {
        k.window = WinCfg{};
        k.window.chunk = t.tile_h;
        k.window.waves = t.waves;
        return win_config(g, method, dtype, k.window);
    }
    if (t.impl == RS_IMPL_REDUCE) return reduce_config(g, method, dtype, src, nullptr);
    if (t.impl == RS_IMPL_STREAM) {
        k.stream = StreamCfg{};
        k.stream.tile_w = t.tile_w;
        k.stream.chunk_h = t.tile_h;
        k.stream.waves = t.waves;
        return stream_config(g, method, dtype, src, k.stream);
    }
    k.tile = TileCfg{t.tile_w, t.tile_h, t.threads, 0, 0, 0};
    return tiled_config(g, method, k.tile);
}

static bool default_choice(const Geom& g, int method, int dtype, const void* src, KernelChoice& k)
{
    if (method == RS_NEAREST) {
        // Strips of 4096 bytes (256 threads across): the staged-rows kernel
        // where its conditions hold, else the per-thread gather.
        const Tuned t{RS_IMPL_GATHER, 256 * (16 / (int)dtype_size(dtype)), nearest_default_rows(g, dtype), 256, 0};
        if (make_choice(g, method, dtype, src, t, k)) return true;
    }
    // Register window for large outputs (a small output has too few strips
    // and bands to fill the GPU) of vertical upscales, and of uint8
    // downscales (measured faster than the streaming kernel there, slower
    // for FP32): 8-row chunks when they leave room for three blocks per SM,
    // else 4-row chunks, within ~100 KB; two blocks per resident slot, one
    // for a single plane's vertical downscale (fewer, longer bands measured
    // faster there).
    const int64_t out_elems = (int64_t)g.Ho * g.Wo * g.C * g.planes;
    // FP32 vertical downscales to at least 1/4 (every source row feeds an
    // output row): the window pass in its transposed roles, within ~100 KB.
    if (dtype == DT_F32 && g.Ho < g.H && 4 * (int64_t)g.Ho >= g.H && out_elems >= (int64_t)1 << 20) {
        size_t smem = 0;
        if (reduce_config(g, method, dtype, src, &smem) && smem <= 100 * 1024) {
            k.impl = RS_IMPL_REDUCE;
            return true;
        }
    }
    if ((g.Ho >= g.H || dtype == DT_U8) && out_elems >= (int64_t)1 << 22) {
        for (int ch : {8, 4}) {
            const Tuned t{RS_IMPL_WINDOW, 1024, ch, 128, g.Ho < g.H && g.planes == 1 ? 1 : 2};
            if (make_choice(g, method, dtype, src, t, k) && k.window.smem <= (ch == 8 ? 56 : 100) * 1024) return true;
        }
    }
    StreamCfg sc = stream_default(g, method, dtype, src);
    if (sc.tile_w) {
        sc.waves = 4;
        k.impl = RS_IMPL_STREAM;
        k.stream = sc;
        return true;
    }
    k.impl = RS_IMPL_TILED;
    k.tile = tiled_default(g, method);
    return k.tile.tile_w != 0;
}

rs_status choose_kernel(const Geom& g, int method, int dtype, const void* src, const rs_options& o,
                        KernelChoice& k)
{
    const bool explicit_shape = o.tile_w || o.tile_h || o.threads || o.waves;
    if (o.impl == RS_IMPL_GATHER) {
        const int ev = 16 / (int)dtype_size(dtype);
        const Tuned t{RS_IMPL_GATHER, o.tile_w ? o.tile_w : 256 * ev, o.tile_h ? o.tile_h : nearest_default_rows(g, dtype),
                      256, 0};
        if (method != RS_NEAREST) return RS_ERR_INVALID_ARG;
        return make_choice(g, method, dtype, src, t, k) ? RS_OK : RS_ERR_INVALID_ARG;
    }
    if (o.impl == RS_IMPL_WINDOW) {
        const Tuned t{RS_IMPL_WINDOW, 1024, o.tile_h ? o.tile_h : 8, 128, o.waves ? o.waves : 2};
        return make_choice(g, method, dtype, src, t, k) ? RS_OK : RS_ERR_INVALID_ARG;
    }
    if (o.impl == RS_IMPL_REDUCE) {
        if (explicit_shape) return RS_ERR_INVALID_ARG;
        const Tuned t{RS_IMPL_REDUCE, 0, 0, 256, 0};
        return make_choice(g, method, dtype, src, t, k) ? RS_OK : RS_ERR_INVALID_ARG;
    }
    if (o.impl == RS_IMPL_STREAM || (o.impl == RS_IMPL_AUTO && explicit_shape && !o.threads)) {
        StreamCfg d = stream_default(g, method, dtype, src);
        Tuned t{RS_IMPL_STREAM, o.tile_w ? o.tile_w : (d.tile_w ? d.tile_w : 512),
                o.tile_h ? o.tile_h : (d.chunk_h ? d.chunk_h : 8), 256, o.waves ? o.waves : 4};
        return make_choice(g, method, dtype, src, t, k) ? RS_OK : RS_ERR_INVALID_ARG;
    }
    if (o.impl == RS_IMPL_TILED || (o.impl == RS_IMPL_AUTO && o.threads)) {
        if (explicit_shape) {
            TileCfg d = tiled_default(g, method);
            Tuned t{RS_IMPL_TILED, o.tile_w ? o.tile_w : d.tile_w, o.tile_h ? o.tile_h : d.tile_h,
                    o.threads ? o.threads : d.threads, 0};
            return make_choice(g, method, dtype, src, t, k) ? RS_OK : RS_ERR_INVALID_ARG;
        }
        k.impl = RS_IMPL_TILED;
        k.tile = tiled_default(g, method);
        return k.tile.tile_w ? RS_OK : RS_ERR_UNSUPPORTED;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_env_once();
        auto it = g_tune.find(tune_key(g, method, dtype));
        if (it != g_tune.end() && make_choice(g, method, dtype, src, it->second, k)) return RS_OK;
    }
    return default_choice(g, method, dtype, src, k) ? RS_OK : RS_ERR_UNSUPPORTED;
}

cudaError_t launch_choice(const Geom& g, int method, int dtype, const void* src, void* dst, const KernelChoice& k,
                          cudaStream_t st)
{
    if (k.impl == RS_IMPL_GATHER) return launch_nearest(g, dtype, src, dst, k.gather_w, k.gather_rows, st);
    if (k.impl == RS_IMPL_WINDOW) return launch_win(g, method, dtype, src, dst, k.window, st);
    if (k.impl == RS_IMPL_STREAM) return launch_stream(g, method, dtype, src, dst, k.stream, st);
    if (k.impl == RS_IMPL_REDUCE) return launch_reduce(g, method, dtype, src, dst, st);
    return launch_tiled(g, method, dtype, src, dst, k.tile, st);
}

// Median time in microseconds of one launch, from 3 batches sized to ~2 ms.
static cudaError_t time_choice(const Geom& g, int method, int dtype, const void* src, void* dst,
                               const KernelChoice& k, cudaStream_t st, float* us)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
    float samples[3] = {0, 0, 0};
    int reps = 1;
    for (int it = -1; it < 3 && e == cudaSuccess; ++it) {
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_choice(g, method, dtype, src, dst, k, st);
        cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (it < 0) reps = std::max(1, std::min(50, (int)std::ceil(2.0f / std::max(ms, 1e-3f))));
        else samples[it] = 1000.0f * ms / reps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    std::sort(samples, samples + 3);
    *us = samples[1];
    return cudaSuccess;
}

static Tuned to_tuned(const KernelChoice& k)
{
    if (k.impl == RS_IMPL_GATHER) return Tuned{RS_IMPL_GATHER, k.gather_w, k.gather_rows, 256, 0};
    if (k.impl == RS_IMPL_WINDOW) return Tuned{RS_IMPL_WINDOW, 1024, k.window.chunk, 128, k.window.waves};
    if (k.impl == RS_IMPL_STREAM) return Tuned{RS_IMPL_STREAM, k.stream.tile_w, k.stream.chunk_h, 256, k.stream.waves};
    if (k.impl == RS_IMPL_REDUCE) return Tuned{RS_IMPL_REDUCE, 0, 0, 256, 0};
    return Tuned{RS_IMPL_TILED, k.tile.tile_w, k.tile.tile_h, k.tile.threads, 0};
}

static void fill(rs_tile_config* c, const Tuned& t)
{
    c->impl = t.impl;
    c->tile_w = t.tile_w;
    c->tile_h = t.tile_h;
    c->threads = t.threads;
    c->waves = t.waves;
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_autotune(const void* src, const rs_layout* in, void* dst, const rs_layout* out, rs_dtype dtype,
                      rs_method method, const rs_options* opt, void* stream, rs_tile_config* best)
{
    rs_options o = options_or_default(opt);
    Geom g;
    rs_status s = make_geom(src, in, dst, out, dtype, method, o, g);
    if (s != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<Tuned> cands;
    cands.push_back(Tuned{RS_IMPL_REDUCE, 0, 0, 256, 0});
    for (int ch : {4, 8, 16})
        for (int wv : {1, 2, 4}) cands.push_back(Tuned{RS_IMPL_WINDOW, 1024, ch, 128, wv});
    for (int tw : {128, 256, 512, 1024})
        for (int ch : {4, 8, 16, 32})
            for (int wv : {2, 4, 8}) cands.push_back(Tuned{RS_IMPL_STREAM, tw, ch, 256, wv});
    for (int tw : {128, 256, 512, 1024})
        for (int th : {4, 8, 16, 32, 64})
            for (int nt : {128, 256}) cands.push_back(Tuned{RS_IMPL_TILED, tw, th, nt, 0});
    if (method == RS_NEAREST) {
        const int ev = 16 / (int)dtype_size(dtype);
        for (int nv : {8, 16, 32, 64, 128, 256})
            for (int rows : {1, 2, 4, 8, 16, 32, 64, 128, 256}) cands.push_back(Tuned{RS_IMPL_GATHER, nv * ev, rows, 256, 0});
    }
    KernelChoice def;
    if (!default_choice(g, method, dtype, src, def)) return RS_ERR_UNSUPPORTED;
    float def_us = 0.0f;
    cudaError_t e = time_choice(g, method, dtype, src, dst, def, st, &def_us);
    if (e != cudaSuccess) return cuda_status(e);
    Tuned bestt = to_tuned(def);
    float best_us = def_us;
    int n = 1;
    for (const Tuned& t : cands) {
        KernelChoice k;
        if (!make_choice(g, method, dtype, src, t, k)) continue;
        float us = 0.0f;
        e = time_choice(g, method, dtype, src, dst, k, st, &us);
        if (e != cudaSuccess) return cuda_status(e);
        ++n;
        if (us < best_us) { best_us = us; bestt = t; }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(g, method, dtype)] = bestt;
    }
    if (best) {
        fill(best, bestt);
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
    // Assume 256-byte aligned buffers (as cudaMalloc returns).
    static const char* const aligned = reinterpret_cast<const char*>(256);
    KernelChoice k;
    if ((s = choose_kernel(g, method, dtype, aligned, o, k)) != RS_OK) return s;
    fill(cfg, to_tuned(k));
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
    std::fprintf(f, "# resample-tune v2: key impl tile_w tile_h threads waves\n");
    for (auto& kv : g_tune)
        std::fprintf(f, "%s %d %d %d %d %d\n", kv.first.c_str(), kv.second.impl, kv.second.tile_w,
                     kv.second.tile_h, kv.second.threads, kv.second.waves);
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
