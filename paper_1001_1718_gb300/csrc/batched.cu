// Ragged batch: many images of uneven sizes, each with its own scale,
// channel count and method, resampled by persistent kernels that walk a
// work list in device memory.
//
// The host sorts the images into classes. A bilinear / bicubic image whose
// footprint fits becomes (strip of 1024 output elements, band of output
// rows) items of the register-window kernel, in the class of its (method,
// channel count); any other image (nearest, or too large a footprint)
// becomes output tiles of the tiled kernel, in one class of its own. Each
// class is a contiguous run of image descriptors with an exclusive prefix
// sum of their item counts; descriptors and prefixes go to device memory
// (the caller's workspace, or the library's fixed array for the
// no-allocation entry point). Each non-empty class is ONE persistent launch,
// fully specialised for its class: one block per resident slot (SM count x
// blocks per SM); block b takes items b, b + gridDim.x, ..., finds each
// item's image by binary search in the class prefix and runs the image's
// per-block work. No block waits on another. The replayable plan records the
// class launches as independent nodes of one CUDA graph. With
// RS_FLAG_ANTIALIAS every image is resampled with the antialias taps: window
// items up to 8 taps per axis, many-tap tiles beyond.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <map>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "win_body.cuh"
#include "tile_body.cuh"
#include "aa_wide.cuh"

namespace rs {

struct BatchImage {
    const void* src;
    void* dst;
    int64_t src_pitch, dst_pitch;
    int H, W, Ho, Wo;
    int C, method, tiles_x, kind;          // tiles_x: items per row of items; kind 0 tile, 1 window, 2 many-tap
    int tile_w, tile_h, sh_max, swe_max;   // kind 0: tiled-kernel tile
    int chunk, band_h, swe, raw_row, band_cap, pos_cap, tab_off, raw_off;   // kind 1: window config
    int aa, strip;                         // antialias taps: the stretched method (0: point taps), window strip
    int KX, KY, TH, RG, fw, nr, s_off, pad;   // kind 2: many-tap antialias tiles (AaWideCfg)
};

// Classes: 0..7 = window (KT 2 / 4) x (C 1..4) with a footprint of at most
// kWindowSmallSmem bytes of shared memory (three blocks per SM), 8..15 the
// same with larger footprints (up to ~100 KB, two blocks per SM), 16 =
// tiled. Splitting by footprint keeps one large image from lowering the
// occupancy of its whole class. With RS_FLAG_ANTIALIAS (the whole batch)
// the window classes hold antialias taps, at most K = 4 / 8 per axis in
// place of KT = 2 / 4, and class 16 the many-tap antialias tiles.
static constexpr int kClasses = 17;
static constexpr int kTileClass = 16;
static constexpr size_t kWindowSmallSmem = 72 * 1024;
static constexpr int kHeavyBand = 32;   // band rows of large-footprint and downscaled window items

__device__ __forceinline__ int find_image(const int64_t* __restrict__ start, int n, int64_t t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ Geom image_geom(const BatchImage& im, int coord, float a)
{
    Geom g;
    g.H = im.H; g.W = im.W; g.Ho = im.Ho; g.Wo = im.Wo; g.C = im.C;
    g.src_pitch = im.src_pitch;
    g.dst_pitch = im.dst_pitch;
    g.sp = PlaneMap{0, 0, 1};
    g.dp = PlaneMap{0, 0, 1};
    g.planes = 1;
    g.coord = coord;
    g.a = a;
    return g;
}

// Window items of one (KT, C) class: point taps (TM = TAP_POINT, KT = the
// method's taps) or antialias taps (TM = TAP_AA, at most KT per axis).
template <int KT, int C, typename T, int TM = TAP_POINT>
__global__ void __launch_bounds__(kWinThreads, 2)
k_batched_window(const BatchImage* __restrict__ imgs, const int64_t* __restrict__ start, int n, int64_t total,
                 int coord, float a, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int k = find_image(start, n, t);
        const BatchImage im = imgs[k];
        const int64_t local = t - __ldg(start + k);
        if (local < 0 || local >= __ldg(start + k + 1) - __ldg(start + k) || im.kind != 1 || im.C != C) {
            if (threadIdx.x == 0) report_fault(fault, FAULT_BATCH_INDEX);   // uniform over the block
            continue;
        }
        const Geom g = image_geom(im, coord, a);
        WinCfg wc;
        wc.chunk = im.chunk;
        wc.band_h = im.band_h;
        wc.waves = 0;
        wc.swe = im.swe;
        wc.raw_row = im.raw_row;
        wc.band_cap = im.band_cap;
        wc.pos_cap = im.pos_cap;
        wc.tab_off = im.tab_off;
        wc.raw_off = im.raw_off;
        wc.aa_method = im.aa;
        wc.strip = im.strip;
        wc.smem = 0;
        win_body<KT, C, T, T, false, TM>(g, static_cast<const T*>(im.src), static_cast<T*>(im.dst), wc,
                                         (int)(local % im.tiles_x), (int)(local / im.tiles_x), sm, fault);
        __syncthreads();   // the next item reuses shared memory
    }
}

// Many-tap antialias tiles (kind 2) of any channel count.
template <typename T>
__global__ void __launch_bounds__(kAwNT)
k_batched_aa_wide(const BatchImage* __restrict__ imgs, const int64_t* __restrict__ start, int n, int64_t total,
                  int coord, float a, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int k = find_image(start, n, t);
        const BatchImage im = imgs[k];
        const int64_t local = t - __ldg(start + k);
        if (local < 0 || local >= __ldg(start + k + 1) - __ldg(start + k) || im.kind != 2) {
            if (threadIdx.x == 0) report_fault(fault, FAULT_BATCH_INDEX);   // uniform over the block
            continue;
        }
        const Geom g = image_geom(im, coord, a);
        AaWideCfg c;
        c.KX = im.KX; c.KY = im.KY; c.TH = im.TH; c.RG = im.RG;
        c.fw = im.fw; c.nr = im.nr; c.method = im.aa; c.s_off = im.s_off;
        c.smem = 0;
        const T* s = static_cast<const T*>(im.src);
        T* d = static_cast<T*>(im.dst);
        const int bx = (int)(local % im.tiles_x), by = (int)(local / im.tiles_x);
        switch (im.C) {
        case 1: aa_wide_body<1, T, T, false>(g, s, d, c, bx, by, sm, fault, NormOut{}); break;
        case 2: aa_wide_body<2, T, T, false>(g, s, d, c, bx, by, sm, fault, NormOut{}); break;
        case 3: aa_wide_body<3, T, T, false>(g, s, d, c, bx, by, sm, fault, NormOut{}); break;
        default: aa_wide_body<4, T, T, false>(g, s, d, c, bx, by, sm, fault, NormOut{}); break;
        }
        __syncthreads();   // the next tile reuses shared memory
    }
}

template <int KT, typename T>
__device__ __forceinline__ void batch_tile_c(const Geom& g, const BatchImage& im, const TileCfg& cfg, int bx,
                                             int by, float* sm, unsigned int* fault)
{
    const T* s = static_cast<const T*>(im.src);
    T* d = static_cast<T*>(im.dst);
    switch (im.C) {
    case 1: tile_body<KT, 1, T>(g, s, d, cfg, bx, by, sm, fault); break;
    case 2: tile_body<KT, 2, T>(g, s, d, cfg, bx, by, sm, fault); break;
    case 3: tile_body<KT, 3, T>(g, s, d, cfg, bx, by, sm, fault); break;
    default: tile_body<KT, 4, T>(g, s, d, cfg, bx, by, sm, fault); break;
    }
}

// Tile items of any method and channel count.
template <typename T>
__global__ void __launch_bounds__(256)
k_batched(const BatchImage* __restrict__ imgs, const int64_t* __restrict__ start, int n, int64_t total,
          int coord, float a, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int k = find_image(start, n, t);
        const BatchImage im = imgs[k];
        const int64_t local = t - __ldg(start + k);
        if (local < 0 || local >= __ldg(start + k + 1) - __ldg(start + k) || im.kind != 0) {
            if (threadIdx.x == 0) report_fault(fault, FAULT_BATCH_INDEX);   // uniform over the block
            continue;
        }
        const Geom g = image_geom(im, coord, a);
        TileCfg cfg;
        cfg.tile_w = im.tile_w;
        cfg.tile_h = im.tile_h;
        cfg.threads = blockDim.x;
        cfg.sh_max = im.sh_max;
        cfg.swe_max = im.swe_max;
        cfg.smem = 0;
        const int bx = (int)(local % im.tiles_x), by = (int)(local / im.tiles_x);
        switch (im.method) {
        case M_NEAREST: batch_tile_c<1, T>(g, im, cfg, bx, by, sm, fault); break;
        case M_BILINEAR: batch_tile_c<2, T>(g, im, cfg, bx, by, sm, fault); break;
        default: batch_tile_c<4, T>(g, im, cfg, bx, by, sm, fault); break;
        }
        __syncthreads();   // the next tile reuses shared memory
    }
}

// ---------------------------------------------------------------------------
// Host side

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
static bool dim_ok(int v) { return v >= 1 && v <= 65535; }

// Tile shape of one image: tile_w elements, the tallest tile_h <= h_cap that
// fits `budget` bytes of shared memory, else the tallest that fits at all.
static bool image_tile(const Geom& g, int method, int tile_w, int h_cap, int threads, size_t budget, TileCfg& out)
{
    for (int pass = 0; pass < 2; ++pass) {
        for (int th = h_cap; th >= 1; th >>= 1) {
            TileCfg c{tile_w, th, threads, 0, 0, 0};
            if (!tiled_config(g, method, c)) continue;
            if (pass == 0 && c.smem > budget) continue;
            out = c;
            return true;
        }
    }
    return false;
}

// Shape of a batch's items: every image as tiles, or bilinear / bicubic
// images as register-window items of `band` output rows whose source rows
// are staged `chunk` at a time (chunk 0: 8, else 4 when 8 does not fit).
struct BatchShape {
    bool tiled;
    int chunk, band;
};

// Antialias taps (RS_FLAG_ANTIALIAS): window items with at most K = 4 or 8
// taps per axis, in the class of (K, C, footprint tier); else (more taps,
// or every image when the batch is tiled) many-tap tiles in the tile class.
static rs_status prepare_image_aa(const rs_image_desc& x, const Geom& g, int dtype, const BatchShape& sh,
                                  BatchImage& im, int& cls, int64_t& items, size_t& smem)
{
    if (x.method != RS_BILINEAR && x.method != RS_BICUBIC) return RS_ERR_INVALID_ARG;
    im.aa = x.method == RS_BILINEAR ? M_BILINEAR : M_BICUBIC;
    const int k = antialias_taps(g, im.aa);
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : 0;
    // chunks of 8 staged rows, else 4 (K = 4), else 16, within the
    // small-footprint budget; else the same within ~100 KB
    const int chunks[3] = {sh.chunk ? sh.chunk : 8, sh.chunk ? 0 : 4, sh.chunk ? 0 : 16};
    for (int t = 0; K && !sh.tiled && t < 6; ++t) {
        const int ch = chunks[t % 3];
        if (!ch || ch % K) continue;
        WinCfg wc{};
        wc.chunk = ch;
        if (!win_config_aa(g, im.aa, dtype, K, wc) || wc.smem > (t < 3 ? kWindowSmallSmem : 100 * 1024)) continue;
        im.kind = 1;
        im.chunk = wc.chunk;
        const bool heavy = t >= 3 || x.Ho < x.H;
        im.band_h = std::min(wc.band_cap, heavy ? std::min(sh.band, kHeavyBand) : sh.band);
        im.swe = wc.swe;
        im.band_cap = wc.band_cap;
        im.pos_cap = wc.pos_cap;
        im.tab_off = wc.tab_off;
        im.raw_row = wc.raw_row;
        im.raw_off = wc.raw_off;
        im.strip = wc.strip;
        im.tiles_x = (int)(((int64_t)x.Wo + wc.strip - 1) / wc.strip);
        items = (int64_t)im.tiles_x * ((x.Ho + im.band_h - 1) / im.band_h);
        smem = wc.smem;
        cls = (wc.smem <= kWindowSmallSmem ? 0 : 8) + (K == 4 ? 0 : 4) + (x.C - 1);
        return RS_OK;
    }
    AaWideCfg c;
    if (!aa_wide_config(g, im.aa, c)) return RS_ERR_UNSUPPORTED;
    im.kind = 2;
    im.KX = c.KX; im.KY = c.KY; im.TH = c.TH; im.RG = c.RG;
    im.fw = c.fw; im.nr = c.nr; im.s_off = c.s_off;
    im.tiles_x = (x.Wo + 31) / 32;
    items = (int64_t)im.tiles_x * ((x.Ho + c.TH - 1) / c.TH);
    smem = c.smem;
    cls = kTileClass;
    return RS_OK;
}

// Validates one descriptor and fills its device descriptor: window items
// (bilinear / bicubic, footprint within ~100 KB of shared memory) or tiles.
// Returns the class, item count and shared-memory need.
static rs_status prepare_image(const rs_image_desc& x, int dtype, const rs_options& o, const BatchShape& sh,
                               int tile_w, int h_cap, int threads, BatchImage& im, int& cls, int64_t& items,
                               size_t& smem)
{
    const int64_t es = (int64_t)dtype_size(dtype);
    if (!x.src || !x.dst) return RS_ERR_INVALID_ARG;
    if (!dim_ok(x.H) || !dim_ok(x.W) || !dim_ok(x.Ho) || !dim_ok(x.Wo)) return RS_ERR_INVALID_ARG;
    if (x.C < 1 || x.C > 4) return RS_ERR_INVALID_ARG;
    if (x.method < RS_NEAREST || x.method > RS_BICUBIC) return RS_ERR_INVALID_ARG;
    if (x.src_pitch < (int64_t)x.W * x.C || x.dst_pitch < (int64_t)x.Wo * x.C) return RS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(x.src) % es || reinterpret_cast<uintptr_t>(x.dst) % es)
        return RS_ERR_ALIGNMENT;
    Geom g;
    g.H = x.H; g.W = x.W; g.Ho = x.Ho; g.Wo = x.Wo; g.C = x.C;
    g.src_pitch = x.src_pitch; g.dst_pitch = x.dst_pitch;
    g.sp = PlaneMap{0, 0, 1}; g.dp = PlaneMap{0, 0, 1};
    g.planes = 1; g.coord = o.coord; g.a = o.cubic_a;
    std::memset(&im, 0, sizeof im);
    im.src = x.src; im.dst = x.dst;
    im.src_pitch = x.src_pitch; im.dst_pitch = x.dst_pitch;
    im.H = x.H; im.W = x.W; im.Ho = x.Ho; im.Wo = x.Wo; im.C = x.C; im.method = x.method;
    if (o.flags & RS_FLAG_ANTIALIAS) return prepare_image_aa(x, g, dtype, sh, im, cls, items, smem);
    if (x.method != RS_NEAREST && !sh.tiled) {
        // chunks of 8 rows, else 4, within the small-footprint budget; else
        // the same within ~100 KB (the large-footprint classes)
        const int chunks[4] = {sh.chunk ? sh.chunk : 8, sh.chunk ? 0 : 4, sh.chunk ? sh.chunk : 8, sh.chunk ? 0 : 4};
        for (int t = 0; t < 4; ++t) {
            const int ch = chunks[t];
            if (!ch) continue;
            WinCfg wc{};
            wc.chunk = ch;
            // the general window body (the batch has no exact-x2 form: one kernel per class)
            if (!win_config(g, x.method, dtype, wc, false) || wc.smem > (t < 2 ? kWindowSmallSmem : 100 * 1024)) continue;
            im.kind = 1;
            im.chunk = wc.chunk;
            // A large footprint or a vertical downscale makes each band row
            // costly (more source rows staged per output row): short bands
            // spread such images over many blocks instead of a few long ones.
            const bool heavy = t >= 2 || x.Ho < x.H;
            im.band_h = std::min(wc.band_cap, heavy ? std::min(sh.band, kHeavyBand) : sh.band);
            im.swe = wc.swe;
            im.band_cap = wc.band_cap;
            im.pos_cap = wc.pos_cap;
            im.tab_off = wc.tab_off;
            im.raw_row = wc.raw_row;
            im.raw_off = wc.raw_off;
            const int sp = kWinThreads * win_pixels(x.C, dtype, false);
            im.tiles_x = (int)(((int64_t)x.Wo + sp - 1) / sp);
            items = (int64_t)im.tiles_x * ((x.Ho + im.band_h - 1) / im.band_h);
            smem = wc.smem;
            cls = (wc.smem <= kWindowSmallSmem ? 0 : 8) + (x.method == RS_BILINEAR ? 0 : 4) + (x.C - 1);
            return RS_OK;
        }
    }
    TileCfg c;
    if (!image_tile(g, x.method, tile_w, h_cap, threads, 72 * 1024, c)) return RS_ERR_UNSUPPORTED;
    im.kind = 0;
    im.tile_w = c.tile_w; im.tile_h = c.tile_h; im.sh_max = c.sh_max; im.swe_max = c.swe_max;
    im.tiles_x = (int)(((int64_t)x.Wo * x.C + c.tile_w - 1) / c.tile_w);
    items = (int64_t)im.tiles_x * ((x.Ho + c.tile_h - 1) / c.tile_h);
    smem = c.smem;
    cls = kTileClass;
    return RS_OK;
}

// Items of one image (as prepare_image counts them) and a rough cost of one
// item: its output rows and the source rows they stage (per strip or tile
// column), plus a fixed part for the block's prologue.
static int64_t image_items(const BatchImage& im)
{
    const int rows = im.kind == 1 ? im.band_h : im.kind == 2 ? im.TH : im.tile_h;
    return (int64_t)im.tiles_x * ((im.Ho + rows - 1) / rows);
}

static double item_cost(const BatchImage& im)
{
    const int rows = im.kind == 1 ? im.band_h : im.kind == 2 ? im.TH : im.tile_h;
    return rows * (1.0 + 0.55 * (double)im.H / (double)im.Ho) + 24.0;
}

// Work-list layout shared by the workspace and the fixed-array paths:
// descriptors grouped by class (class c occupies [first[c], first[c] +
// count[c])), then per class an exclusive prefix of count[c] + 1 entries
// starting at prefix[c] (an index into the int64 prefix area).
struct BatchLayout {
    int count[kClasses], first[kClasses], prefix[kClasses];
    int64_t total[kClasses];
    size_t smem[kClasses];
    double item_cost[kClasses];   // mean cost of the class's items (item_cost)
    int threads;
    int n;
};

// Fills imgs_out (n entries) and start_out (n + kClasses entries) grouped
// by class, with no allocation (scratch arrays are caller-provided, n each).
// Tuning-cache key of a batch: GPU (model, CUDA runtime, SM count), dtype,
// count, coordinate map and a hash of every descriptor's sizes, channels,
// method and pitches.
static std::string batch_key(const rs_image_desc* d, int n, int dtype, const rs_options& o)
{
    uint64_t h = 1469598103934665603ull;   // FNV-1a
    auto mix = [&](int64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)(v >> (8 * i)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    for (int k = 0; k < n; ++k) {
        mix(d[k].H); mix(d[k].W); mix(d[k].C); mix(d[k].Ho); mix(d[k].Wo);
        mix(d[k].method); mix(d[k].src_pitch); mix(d[k].dst_pitch);
    }
    char buf[96];
    std::snprintf(buf, sizeof buf, ";sms=%d;batch;dt=%d;n=%d;coord=%d;aa=%d;h=%016llx", num_sms(), dtype, n, o.coord,
                  (int)(o.flags & RS_FLAG_ANTIALIAS), (unsigned long long)h);
    return "gpu=" + device_tag() + buf;
}

// Item shape from the options: RS_IMPL_TILED (or an explicit tile shape with
// RS_IMPL_AUTO) tiles every image; RS_IMPL_WINDOW takes band = tile_w
// (default 256) and chunk = tile_h (default 0); RS_IMPL_AUTO takes the
// tuned shape of this batch when the cache has one (`tuned`), else the
// default window shape. Other kernels have no batched form.
static rs_status batch_shape(const rs_image_desc* d, int n, int dtype, const rs_options& o, bool tuned,
                             BatchShape& sh)
{
    const bool explicit_shape = o.tile_w || o.tile_h || o.threads;
    if (o.impl == RS_IMPL_TILED || (o.impl == RS_IMPL_AUTO && explicit_shape)) {
        sh = BatchShape{true, 0, 0};
        return RS_OK;
    }
    if (o.impl == RS_IMPL_WINDOW) {
        sh = BatchShape{false, o.tile_h, o.tile_w ? o.tile_w : kWinMaxBand};
        if (sh.chunk && (sh.chunk < 4 || sh.chunk > 32)) return RS_ERR_INVALID_ARG;
        if (sh.band < 1 || sh.band > kWinMaxBand) return RS_ERR_INVALID_ARG;
        return RS_OK;
    }
    if (o.impl != RS_IMPL_AUTO) return RS_ERR_INVALID_ARG;
    sh = BatchShape{false, 0, kWinMaxBand};
    Tuned t;
    if (tuned && tune_lookup(batch_key(d, n, dtype, o), t)) {
        if (t.impl == RS_IMPL_TILED) sh = BatchShape{true, 0, 0};
        else if (t.impl == RS_IMPL_WINDOW && t.tile_w >= 1 && t.tile_w <= kWinMaxBand) sh = BatchShape{false, t.tile_h, t.tile_w};
    }
    return RS_OK;
}

static rs_status batch_layout(const rs_image_desc* d, int n, int dtype, const rs_options& o, bool tuned,
                              BatchImage* imgs_out, int64_t* start_out, BatchImage* tmp_imgs, int* tmp_cls,
                              int64_t* tmp_items, BatchLayout& L)
{
    if (!d || n < 1) return RS_ERR_INVALID_ARG;
    if (dtype < RS_U8 || dtype > RS_F32) return RS_ERR_INVALID_ARG;
    rs_status s = check_options(o, RS_BILINEAR);
    if (s != RS_OK) return s;
    if (o.flags & ~RS_FLAG_ANTIALIAS) return RS_ERR_INVALID_ARG;
    BatchShape sh;
    if ((s = batch_shape(d, n, dtype, o, tuned, sh)) != RS_OK) return s;
    const bool window_opts = o.impl == RS_IMPL_WINDOW;   // tile_w / tile_h describe the window items
    const int tile_w = o.tile_w && !window_opts ? o.tile_w : 512;
    const int h_cap = o.tile_h && !window_opts ? o.tile_h : 32;
    L.threads = o.threads ? o.threads : 256;
    if (L.threads != 128 && L.threads != 256) return RS_ERR_INVALID_ARG;
    L.n = n;
    for (int c = 0; c < kClasses; ++c) { L.count[c] = 0; L.total[c] = 0; L.smem[c] = 0; }
    const int64_t es = (int64_t)dtype_size(dtype);
    for (int k = 0; k < n; ++k) {
        size_t sm = 0;
        s = prepare_image(d[k], dtype, o, sh, tile_w, h_cap, L.threads, tmp_imgs[k], tmp_cls[k], tmp_items[k], sm);
        if (s != RS_OK) return s;
        L.count[tmp_cls[k]]++;
        L.smem[tmp_cls[k]] = std::max(L.smem[tmp_cls[k]], sm);
    }
    // No destination may overlap any source or another destination.
    auto src_bytes = [&](const rs_image_desc& x) { return ((int64_t)(x.H - 1) * x.src_pitch + (int64_t)x.W * x.C) * es; };
    auto dst_bytes = [&](const rs_image_desc& x) { return ((int64_t)(x.Ho - 1) * x.dst_pitch + (int64_t)x.Wo * x.C) * es; };
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            if (overlaps(d[k].dst, dst_bytes(d[k]), d[l].src, src_bytes(d[l]))) return RS_ERR_INVALID_ARG;
            if (l != k && overlaps(d[k].dst, dst_bytes(d[k]), d[l].dst, dst_bytes(d[l]))) return RS_ERR_INVALID_ARG;
        }
    int first = 0, pre = 0;
    for (int c = 0; c < kClasses; ++c) {
        L.first[c] = first;
        L.prefix[c] = pre;
        first += L.count[c];
        pre += L.count[c] + 1;
    }
    int fill[kClasses];
    for (int c = 0; c < kClasses; ++c) {
        fill[c] = 0;
        start_out[L.prefix[c]] = 0;
    }
    for (int k = 0; k < n; ++k) {
        const int c = tmp_cls[k];
        imgs_out[L.first[c] + fill[c]++] = tmp_imgs[k];
    }
    // Within a class, images with the costliest items first: block b takes
    // items b, b + grid, ..., so neighbouring items of similar cost spread
    // evenly over the blocks and the launch ends with the cheap ones.
    for (int c = 0; c < kClasses; ++c) {
        BatchImage* first = imgs_out + L.first[c];
        std::sort(first, first + L.count[c], [](const BatchImage& a, const BatchImage& b) {
            const double ka = item_cost(a), kb = item_cost(b);
            if (ka != kb) return ka > kb;
            return a.H * (int64_t)a.W < b.H * (int64_t)b.W;
        });
        int64_t* st = start_out + L.prefix[c];
        double cost = 0.0;
        for (int pos = 0; pos < L.count[c]; ++pos) {
            const int64_t it = image_items(first[pos]);
            st[pos + 1] = st[pos] + it;
            cost += item_cost(first[pos]) * (double)it;
        }
        L.item_cost[c] = st[L.count[c]] > 0 ? cost / (double)st[L.count[c]] : 0.0;
    }
    for (int c = 0; c < kClasses; ++c) L.total[c] = start_out[L.prefix[c] + L.count[c]];
    return RS_OK;
}

template <int KT, int C, typename T, int TM = TAP_POINT>
static void* win_func() { return reinterpret_cast<void*>(&k_batched_window<KT, C, T, TM>); }

// Antialias classes: (c & 4) ? 8 : 4 taps per axis, C = (c & 3) + 1; the
// tile class holds the many-tap tiles.
template <typename T>
static void* class_func_aa(int c)
{
    if (c == kTileClass) return reinterpret_cast<void*>(&k_batched_aa_wide<T>);
    switch (c & 7) {
    case 0: return win_func<4, 1, T, TAP_AA>();
    case 1: return win_func<4, 2, T, TAP_AA>();
    case 2: return win_func<4, 3, T, TAP_AA>();
    case 3: return win_func<4, 4, T, TAP_AA>();
    case 4: return win_func<8, 1, T, TAP_AA>();
    case 5: return win_func<8, 2, T, TAP_AA>();
    case 6: return win_func<8, 3, T, TAP_AA>();
    default: return win_func<8, 4, T, TAP_AA>();
    }
}

template <typename T>
static void* class_func_t(int c, bool aa)
{
    if (aa) return class_func_aa<T>(c);
    if (c == kTileClass) return reinterpret_cast<void*>(&k_batched<T>);
    switch (c & 7) {
    case 0: return win_func<2, 1, T>();
    case 1: return win_func<2, 2, T>();
    case 2: return win_func<2, 3, T>();
    case 3: return win_func<2, 4, T>();
    case 4: return win_func<4, 1, T>();
    case 5: return win_func<4, 2, T>();
    case 6: return win_func<4, 3, T>();
    default: return win_func<4, 4, T>();
    }
}

static void* class_func(int dtype, int c, bool aa)
{
    switch (dtype) {
    case DT_U8: return class_func_t<uint8_t>(c, aa);
    case DT_F16: return class_func_t<__half>(c, aa);
    case DT_BF16: return class_func_t<__nv_bfloat16>(c, aa);
    default: return class_func_t<float>(c, aa);
    }
}

// Launch parameters of one class (kernel arguments live in the struct so a
// graph node can point at them while it is created).
struct ClassLaunch {
    void* func;
    dim3 grid, block;
    size_t smem;
    const BatchImage* imgs;
    const int64_t* start;
    int n;
    int64_t total;
    int coord;
    float a;
    unsigned int* fault;
};

static cudaError_t class_launches(const BatchLayout& L, int dtype, const rs_options& o, const void* imgs_dev,
                                  const void* start_dev, ClassLaunch* out, int& nl)
{
    // Classes with the costliest items first: each next class fills the SMs
    // as the previous one's blocks finish, and the step ends on the finest
    // items.
    int order[kClasses];
    for (int c = 0; c < kClasses; ++c) {   // insertion sort, stable
        int k = c;
        while (k > 0 && L.item_cost[order[k - 1]] < L.item_cost[c]) {
            order[k] = order[k - 1];
            --k;
        }
        order[k] = c;
    }
    nl = 0;
    for (int oi = 0; oi < kClasses; ++oi) {
        const int c = order[oi];
        if (L.count[c] == 0 || L.total[c] == 0) continue;
        ClassLaunch& cl = out[nl++];
        const bool aa = (o.flags & RS_FLAG_ANTIALIAS) != 0;
        cl.func = class_func(dtype, c, aa);
        const int threads = c == kTileClass ? (aa ? kAwNT : L.threads) : kWinThreads;
        int per_sm = 0;
        cudaError_t e = prepare_kernel(cl.func, L.smem[c], threads, &per_sm);
        if (e != cudaSuccess) return e;
        const int64_t blocks = std::min<int64_t>(L.total[c], (int64_t)num_sms() * std::max(1, per_sm));
        cl.grid = dim3((unsigned)std::max<int64_t>(1, blocks));
        cl.block = dim3(threads);
        cl.smem = L.smem[c];
        cl.imgs = static_cast<const BatchImage*>(imgs_dev) + L.first[c];
        cl.start = static_cast<const int64_t*>(start_dev) + L.prefix[c];
        cl.n = L.count[c];
        cl.total = L.total[c];
        cl.coord = o.coord;
        cl.a = o.cubic_a;
        cl.fault = fault_word();
    }
    return cudaSuccess;
}

static cudaError_t launch_classes(ClassLaunch* cls, int nl, cudaStream_t st)
{
    for (int i = 0; i < nl; ++i) {
        ClassLaunch& c = cls[i];
        void* args[] = {&c.imgs, &c.start, &c.n, &c.total, &c.coord, &c.a, &c.fault};
        cudaError_t e = cudaLaunchKernel(c.func, c.grid, c.block, args, c.smem, st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Host-side work list for the workspace entry points.
struct BatchPlanHost {
    std::vector<BatchImage> imgs;
    std::vector<int64_t> start;
    BatchLayout L;
    size_t ws_bytes = 0, off_start = 0;
};

static rs_status batch_prepare(const rs_image_desc* d, int n, int dtype, const rs_options& o, BatchPlanHost& P)
{
    if (!d || n < 1 || n > (1 << 20)) return RS_ERR_INVALID_ARG;
    P.imgs.resize(n);
    P.start.assign((size_t)n + kClasses, 0);
    std::vector<BatchImage> tmp(n);
    std::vector<int> cls(n);
    std::vector<int64_t> items(n);
    rs_status s = batch_layout(d, n, dtype, o, true, P.imgs.data(), P.start.data(), tmp.data(), cls.data(),
                               items.data(), P.L);
    if (s != RS_OK) return s;
    P.off_start = align256(sizeof(BatchImage) * (size_t)n);
    P.ws_bytes = P.off_start + sizeof(int64_t) * P.start.size();
    return RS_OK;
}

static cudaError_t upload(const BatchPlanHost& P, void* ws, cudaStream_t st)
{
    std::vector<char> blob(P.ws_bytes, 0);
    std::memcpy(blob.data(), P.imgs.data(), sizeof(BatchImage) * P.imgs.size());
    std::memcpy(blob.data() + P.off_start, P.start.data(), sizeof(int64_t) * P.start.size());
    cudaError_t e = cudaMemcpyAsync(ws, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    // The host blob dies with this function: wait for the copy to finish.
    return cudaStreamSynchronize(st);
}

static rs_status check_ws(const BatchPlanHost& P, void* ws, size_t bytes)
{
    if (!ws || bytes < P.ws_bytes) return RS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) % 256) return RS_ERR_ALIGNMENT;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// Batched resampling without any allocation.
//
// Some callers cannot obtain device memory for the workspace: code running
// under an allocator that owns all device memory (a framework's caching
// pool or a fixed memory budget), real-time serving paths that forbid any
// allocation after start-up because cudaMalloc can block or fail, and plugin
// hosts that only hand out their own input and output buffers. For them the
// work list lives in a fixed array of device memory that the library itself
// declares (file scope, `static __device__`), so no call allocates: every GPU
// that loads the library holds kNoAllocBytes of it until the process exits.
//
// In host code the array's name is only a host-side handle, not a device
// address; its device address is looked up per device with
// cudaGetSymbolAddress (on the first call made on that device, with that
// device current) and passed to the kernel like any other pointer.
static constexpr int kNoAllocMaxImages = 4096;
static constexpr size_t kNoAllocImgBytes = ((sizeof(BatchImage) * kNoAllocMaxImages + 255) / 256) * 256;
static constexpr size_t kNoAllocBytes = kNoAllocImgBytes + sizeof(int64_t) * (kNoAllocMaxImages + kClasses);
static __device__ __align__(256) unsigned char g_batch_scratch[kNoAllocBytes];

static constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;                               // guards everything below
static void* g_noalloc_dev[kNoAllocMaxDevices];               // device address per device
static BatchImage g_noalloc_imgs[kNoAllocMaxImages];           // host staging (no heap use)
static int64_t g_noalloc_start[kNoAllocMaxImages + kClasses];
static BatchImage g_noalloc_tmp[kNoAllocMaxImages];
static int g_noalloc_cls[kNoAllocMaxImages];
static int64_t g_noalloc_items[kNoAllocMaxImages];

}  // namespace rs

extern "C" rs_status rs_resize_batched_noalloc(const rs_image_desc* d, int n, rs_dtype dtype, const rs_options* opt,
                                               void* stream)
{
    using namespace rs;
    const rs_options o = options_or_default(opt);
    if (!d || n < 1) return RS_ERR_INVALID_ARG;
    if (n > kNoAllocMaxImages) return RS_ERR_WORKSPACE;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    BatchLayout L;
    rs_status s = batch_layout(d, n, dtype, o, false, g_noalloc_imgs, g_noalloc_start, g_noalloc_tmp, g_noalloc_cls,
                               g_noalloc_items, L);
    if (s != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The descriptors are copied from host staging arrays that the next call
    // refills; a captured copy would replay whatever they hold by then.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_status(e);
    if (cap != cudaStreamCaptureStatusNone) return RS_ERR_UNSUPPORTED;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RS_ERR_UNSUPPORTED;
    if (!g_noalloc_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();   // leave no sticky error for a later, unrelated check
            return cuda_status(e);
        }
        g_noalloc_dev[dev] = p;
    }
    char* scratch = static_cast<char*>(g_noalloc_dev[dev]);
    // Pageable source: each copy returns once the host data has been staged,
    // so the staging arrays may be refilled by the next call.
    e = cudaMemcpyAsync(scratch, g_noalloc_imgs, sizeof(BatchImage) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kNoAllocImgBytes, g_noalloc_start, sizeof(int64_t) * (size_t)(n + kClasses),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    ClassLaunch cls[kClasses];
    int nl = 0;
    if ((e = class_launches(L, dtype, o, scratch, scratch + kNoAllocImgBytes, cls, nl)) != cudaSuccess)
        return cuda_status(e);
    return cuda_status(launch_classes(cls, nl, st));
}

using namespace rs;

struct rs_batched_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    int kernels = 0;   // kernel launches per replay (one per non-empty class)
};

extern "C" {

rs_status rs_resize_batched_workspace(const rs_image_desc* d, int n, rs_dtype dtype, size_t* bytes)
{
    if (!bytes) return RS_ERR_INVALID_ARG;
    rs_options o;
    rs_options_init(&o);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    *bytes = P.ws_bytes;
    return RS_OK;
}

rs_status rs_resize_batched(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace, size_t workspace_bytes,
                            const rs_options* opt, void* stream)
{
    const rs_options o = options_or_default(opt);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    if ((s = check_ws(P, workspace, workspace_bytes)) != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(P, workspace, st);
    if (e != cudaSuccess) return cuda_status(e);
    ClassLaunch cls[kClasses];
    int nl = 0;
    if ((e = class_launches(P.L, dtype, o, workspace, static_cast<char*>(workspace) + P.off_start, cls, nl)) !=
        cudaSuccess)
        return cuda_status(e);
    return cuda_status(launch_classes(cls, nl, st));
}

rs_status rs_batched_plan_create(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace,
                                 size_t workspace_bytes, const rs_options* opt, void* stream, rs_batched_plan** plan)
{
    if (!plan) return RS_ERR_INVALID_ARG;
    *plan = nullptr;
    const rs_options o = options_or_default(opt);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    if ((s = check_ws(P, workspace, workspace_bytes)) != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(P, workspace, st);
    if (e != cudaSuccess) return cuda_status(e);
    ClassLaunch cls[kClasses];
    int nl = 0;
    if ((e = class_launches(P.L, dtype, o, workspace, static_cast<char*>(workspace) + P.off_start, cls, nl)) !=
        cudaSuccess)
        return cuda_status(e);

    rs_batched_plan* p = new rs_batched_plan();
    cudaGetDevice(&p->device);
    e = cudaGraphCreate(&p->graph, 0);
    // One kernel node per class, with no dependencies between them: the
    // class launches may run concurrently.
    for (int i = 0; i < nl && e == cudaSuccess; ++i) {
        ClassLaunch& c = cls[i];
        void* args[] = {&c.imgs, &c.start, &c.n, &c.total, &c.coord, &c.a, &c.fault};
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.func = c.func;
        kp.gridDim = c.grid;
        kp.blockDim = c.block;
        kp.sharedMemBytes = (unsigned)c.smem;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, p->graph, nullptr, 0, &kp);
    }
    p->kernels = nl;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return cuda_status(e);
    }
    *plan = p;
    return RS_OK;
}

rs_status rs_batched_plan_launch(rs_batched_plan* plan, void* stream)
{
    if (!plan || !plan->exec) return RS_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
}

rs_status rs_batched_plan_kernels(const rs_batched_plan* plan, int32_t* kernels)
{
    if (!plan || !kernels) return RS_ERR_INVALID_ARG;
    *kernels = plan->kernels;
    return RS_OK;
}

rs_status rs_batched_plan_destroy(rs_batched_plan* plan)
{
    if (!plan) return RS_ERR_INVALID_ARG;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return RS_OK;
}

rs_status rs_autotune_batched(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace,
                              size_t workspace_bytes, const rs_options* opt, void* stream, rs_tile_config* best)
{
    if (!best) return RS_ERR_INVALID_ARG;
    rs_options o = options_or_default(opt);
    o.impl = RS_IMPL_AUTO;
    o.tile_w = o.tile_h = o.threads = o.waves = 0;
    struct Cand {
        int impl, band, chunk;
    };
    // The default shape first, then band heights x chunk heights, then tiles.
    const Cand cands[] = {{RS_IMPL_WINDOW, 256, 0}, {RS_IMPL_WINDOW, 128, 0}, {RS_IMPL_WINDOW, 64, 0},
                          {RS_IMPL_WINDOW, 32, 0},  {RS_IMPL_WINDOW, 256, 4}, {RS_IMPL_WINDOW, 128, 4},
                          {RS_IMPL_WINDOW, 64, 4},  {RS_IMPL_TILED, 0, 0}};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    rs_status result = RS_OK;
    float best_us = 0.0f, default_us = 0.0f;
    int best_i = -1, timed = 0;
    for (int i = 0; i < (int)(sizeof cands / sizeof cands[0]) && e == cudaSuccess; ++i) {
        rs_options oc = o;
        oc.impl = cands[i].impl;
        oc.tile_w = cands[i].band;
        oc.tile_h = cands[i].chunk;
        BatchPlanHost P;
        rs_status s = batch_prepare(d, n, dtype, oc, P);
        if (s == RS_OK) s = check_ws(P, workspace, workspace_bytes);
        if (s != RS_OK) {
            if (i == 0) { result = s; break; }   // the default shape must be valid
            continue;
        }
        if ((e = upload(P, workspace, st)) != cudaSuccess) break;
        ClassLaunch cls[kClasses];
        int nl = 0;
        if ((e = class_launches(P.L, dtype, oc, workspace, static_cast<char*>(workspace) + P.off_start, cls, nl)) !=
            cudaSuccess)
            break;
        // One untimed launch, then the mean of three.
        if ((e = launch_classes(cls, nl, st)) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) break;
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_classes(cls, nl, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
        if (e != cudaSuccess) break;
        const float us = ms * 1000.0f / 3.0f;
        ++timed;
        if (i == 0) default_us = us;
        if (best_i < 0 || us < best_us) {
            best_i = i;
            best_us = us;
        }
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (e != cudaSuccess) return cuda_status(e);
    if (result != RS_OK) return result;
    const Cand& c = cands[best_i];
    // Tiled batches are stored with the batch's tile defaults (512 x 32).
    const Tuned t = c.impl == RS_IMPL_TILED ? Tuned{RS_IMPL_TILED, 512, 32, 256, 0} : Tuned{c.impl, c.band, c.chunk, 256, 0};
    tune_store(batch_key(d, n, dtype, o), t);
    best->impl = c.impl;
    best->tile_w = c.band;
    best->tile_h = c.chunk;
    best->threads = 256;
    best->waves = 0;
    best->best_us = best_us;
    best->default_us = default_us;
    best->candidates = timed;
    return RS_OK;
}

}  // extern "C"
