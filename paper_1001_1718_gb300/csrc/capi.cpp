// C ABI of libresample: argument validation, layout classification and
// dispatch to the kernels. Nothing is launched unless every argument checks.
#include <cmath>
#include <cstring>

#include "../../include/resample.h"
#include "rs_internal.h"
#include "capi_internal.h"

namespace rs {

thread_local int t_last_cuda_error = 0;

rs_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return RS_OK;
    t_last_cuda_error = (int)e;
    return RS_ERR_CUDA;
}

rs_options options_or_default(const rs_options* opt)
{
    rs_options o;
    rs_options_init(&o);
    if (opt) o = *opt;
    return o;
}

rs_status check_options(const rs_options& o, int method)
{
    if (o.coord < RS_COORD_ASYMMETRIC || o.coord > RS_COORD_ALIGN_CORNERS) return RS_ERR_INVALID_ARG;
    if (!std::isfinite(o.cubic_a)) return RS_ERR_INVALID_ARG;
    if (o.impl < RS_IMPL_AUTO || o.impl > RS_IMPL_REDUCE) return RS_ERR_INVALID_ARG;
    if (o.tile_w < 0 || o.tile_h < 0 || o.threads < 0 || o.waves < 0) return RS_ERR_INVALID_ARG;
    if (o.flags & ~RS_FLAG_ANTIALIAS) return RS_ERR_INVALID_ARG;
    if (method < RS_NEAREST || method > RS_BICUBIC) return RS_ERR_INVALID_ARG;
    return RS_OK;
}

static bool dim_ok(int v) { return v >= 1 && v <= 65535; }

// Classifies a layout. kind: 0 interleaved (C <= 4, incl. C == 1), 1 planar.
rs_status classify(const rs_layout* L, LayoutInfo& info)
{
    if (!L) return RS_ERR_INVALID_ARG;
    if (L->N < 1 || L->C < 1 || !dim_ok(L->H) || !dim_ok(L->W)) return RS_ERR_INVALID_ARG;
    if (L->n_stride < 0 || L->c_stride < 0 || L->row_pitch < 0 || L->px_stride < 1) return RS_ERR_INVALID_ARG;
    if (L->C == 1 || (L->px_stride == L->C && L->c_stride == 1)) {
        if (L->C > 4) return RS_ERR_UNSUPPORTED;
        if (L->px_stride != L->C) return RS_ERR_INVALID_ARG;
        info.kind = 0;
        info.ci = L->C;
        info.cp = 1;
    } else if (L->px_stride == 1) {
        info.kind = 1;
        info.ci = 1;
        info.cp = L->C;
    } else {
        return RS_ERR_UNSUPPORTED;
    }
    const int64_t row_elems = (int64_t)L->W * L->px_stride;
    if (L->row_pitch < row_elems) return RS_ERR_INVALID_ARG;
    const int64_t plane_extent = (int64_t)(L->H - 1) * L->row_pitch + row_elems;
    if (info.cp > 1 && L->c_stride < plane_extent) return RS_ERR_INVALID_ARG;
    const int64_t image_extent = (int64_t)(info.cp - 1) * L->c_stride + plane_extent;
    if (L->N > 1 && L->n_stride < image_extent) return RS_ERR_INVALID_ARG;
    if ((int64_t)L->N * info.cp > 65535) return RS_ERR_UNSUPPORTED;
    info.extent = (int64_t)(L->N - 1) * L->n_stride + image_extent;
    return RS_OK;
}

bool overlaps(const void* a, int64_t abytes, const void* b, int64_t bbytes)
{
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + bbytes && pb < pa + abytes;
}

rs_status geom_from_layouts(const rs_layout* in, const rs_layout* out, int dtype, int method,
                            const rs_options& o, Geom& g, LayoutInfo& li, LayoutInfo& lo)
{
    if (dtype < RS_U8 || dtype > RS_F32) return RS_ERR_INVALID_ARG;
    rs_status s = check_options(o, method);
    if (s != RS_OK) return s;
    if ((s = classify(in, li)) != RS_OK) return s;
    if ((s = classify(out, lo)) != RS_OK) return s;
    if (in->N != out->N || in->C != out->C || li.kind != lo.kind) return RS_ERR_INVALID_ARG;
    g.H = in->H; g.W = in->W; g.Ho = out->H; g.Wo = out->W;
    g.C = li.ci;
    g.src_pitch = in->row_pitch;
    g.dst_pitch = out->row_pitch;
    g.sp = PlaneMap{in->n_stride, in->c_stride, li.cp};
    g.dp = PlaneMap{out->n_stride, out->c_stride, lo.cp};
    g.planes = in->N * li.cp;
    g.coord = o.coord;
    g.a = o.cubic_a;
    return RS_OK;
}

rs_status make_geom(const void* src, const rs_layout* in, const void* dst, const rs_layout* out,
                    int dtype, int method, const rs_options& o, Geom& g)
{
    if (!src || !dst) return RS_ERR_INVALID_ARG;
    LayoutInfo li, lo;
    rs_status s = geom_from_layouts(in, out, dtype, method, o, g, li, lo);
    if (s != RS_OK) return s;
    const size_t es = dtype_size(dtype);
    if (reinterpret_cast<uintptr_t>(src) % es || reinterpret_cast<uintptr_t>(dst) % es)
        return RS_ERR_ALIGNMENT;
    if (overlaps(src, li.extent * (int64_t)es, dst, lo.extent * (int64_t)es)) return RS_ERR_INVALID_ARG;
    return RS_OK;
}

}  // namespace rs

using namespace rs;

extern "C" {

void rs_options_init(rs_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->coord = RS_COORD_ASYMMETRIC;
    opt->cubic_a = -0.5f;
    opt->impl = RS_IMPL_AUTO;
}

rs_layout rs_layout_hwc(int32_t N, int32_t H, int32_t W, int32_t C)
{
    rs_layout L;
    L.N = N; L.C = C; L.H = H; L.W = W;
    L.px_stride = C;
    L.c_stride = 1;
    L.row_pitch = (int64_t)W * C;
    L.n_stride = (int64_t)H * W * C;
    return L;
}

rs_layout rs_layout_nchw(int32_t N, int32_t C, int32_t H, int32_t W)
{
    rs_layout L;
    L.N = N; L.C = C; L.H = H; L.W = W;
    L.px_stride = 1;
    L.row_pitch = W;
    L.c_stride = (int64_t)H * W;
    L.n_stride = (int64_t)C * H * W;
    return L;
}

const char* rs_status_string(rs_status s)
{
    switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_UNSUPPORTED: return "unsupported";
    case RS_ERR_ALIGNMENT: return "misaligned pointer";
    case RS_ERR_WORKSPACE: return "workspace missing or too small";
    case RS_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

const char* rs_version(void) { return "resample-gb300 0.1 (sm_103a)"; }

int rs_last_cuda_error(void) { return t_last_cuda_error; }

rs_status rs_resize_ex(const void* src, const rs_layout* in, void* dst, const rs_layout* out,
                       rs_dtype dtype, rs_method method, const rs_options* opt, void* stream)
{
    const rs_options o = options_or_default(opt);
    Geom g;
    rs_status s = make_geom(src, in, dst, out, dtype, method, o, g);
    if (s != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (o.flags & RS_FLAG_ANTIALIAS) return resize_antialias(g, method, dtype, src, dst, o, st);
    if (o.impl == RS_IMPL_PLAIN) {
        const int bw = o.tile_w ? o.tile_w : 32, bh = o.tile_h ? o.tile_h : 4;
        if (bw * bh > 1024 || bw < 1 || bh < 1 || bh > 64) return RS_ERR_INVALID_ARG;
        return cuda_status(launch_plain(g, method, dtype, src, dst, bw, bh, st));
    }
    KernelChoice k;
    if ((s = choose_kernel(g, method, dtype, src, o, k)) != RS_OK) return s;
    return cuda_status(launch_choice(g, method, dtype, src, dst, k, st));
}

rs_status rs_resize_normalize(const void* src, const rs_layout* in, void* dst, const rs_layout* out,
                              rs_dtype out_dtype, rs_method method, const float* mean, const float* stddev,
                              const rs_options* opt, void* stream)
{
    const rs_options o = options_or_default(opt);
    if (!src || !dst || !mean || !stddev || !in || !out) return RS_ERR_INVALID_ARG;
    if (out_dtype != RS_F16 && out_dtype != RS_BF16 && out_dtype != RS_F32) return RS_ERR_INVALID_ARG;
    rs_status s = check_options(o, method);
    if (s != RS_OK) return s;
    if (method == RS_NEAREST) return RS_ERR_UNSUPPORTED;
    if ((o.impl != RS_IMPL_AUTO && o.impl != RS_IMPL_WINDOW) || o.tile_w || o.threads) return RS_ERR_INVALID_ARG;
    if ((o.flags & RS_FLAG_ANTIALIAS) && o.tile_h) return RS_ERR_INVALID_ARG;
    LayoutInfo li, lo;
    if ((s = classify(in, li)) != RS_OK) return s;
    if ((s = classify(out, lo)) != RS_OK) return s;
    // interleaved source, planar output (for one channel the two coincide)
    if (li.kind != 0 || (in->C > 1 && lo.kind != 1) || in->N != out->N || in->C != out->C) return RS_ERR_INVALID_ARG;
    NormOut no;
    no.c_stride = out->c_stride;
    for (int c = 0; c < 4; ++c) {
        no.scale[c] = 1.0f;
        no.bias[c] = 0.0f;
    }
    for (int c = 0; c < in->C; ++c) {
        if (!std::isfinite(mean[c]) || !std::isfinite(stddev[c]) || stddev[c] == 0.0f) return RS_ERR_INVALID_ARG;
        no.scale[c] = 1.0f / stddev[c];
        no.bias[c] = -mean[c] / stddev[c];
        if (!std::isfinite(no.scale[c]) || !std::isfinite(no.bias[c])) return RS_ERR_INVALID_ARG;
    }
    const size_t eo = dtype_size(out_dtype);
    if (reinterpret_cast<uintptr_t>(dst) % eo) return RS_ERR_ALIGNMENT;
    if (overlaps(src, li.extent, dst, lo.extent * (int64_t)eo)) return RS_ERR_INVALID_ARG;
    Geom g;
    g.H = in->H; g.W = in->W; g.Ho = out->H; g.Wo = out->W;
    g.C = in->C;
    g.src_pitch = in->row_pitch;
    g.dst_pitch = out->row_pitch;
    g.sp = PlaneMap{in->n_stride, 0, 1};
    g.dp = PlaneMap{out->n_stride, 0, 1};
    g.planes = in->N;
    g.coord = o.coord;
    g.a = o.cubic_a;
    if (o.flags & RS_FLAG_ANTIALIAS)
        return resize_normalize_antialias(g, method, out_dtype, src, dst, no, o, static_cast<cudaStream_t>(stream));
    // the window kernel: chunks of 8 staged rows, else 4 (larger footprints)
    WinCfg c{};
    c.waves = o.waves;
    bool ok = false;
    for (int ch : {o.tile_h ? o.tile_h : 8, o.tile_h ? 0 : 4}) {
        if (!ch) continue;
        c.chunk = ch;
        if (win_config(g, method, DT_U8, c)) {
            ok = true;
            break;
        }
    }
    if (!ok) return o.tile_h ? RS_ERR_INVALID_ARG : RS_ERR_UNSUPPORTED;
    return cuda_status(launch_win_norm(g, method, out_dtype, src, dst, c, no, static_cast<cudaStream_t>(stream)));
}

rs_status rs_resize(const void* src, int H, int W, int C, rs_dtype dtype, void* dst, int Ho, int Wo,
                    rs_method method, void* stream)
{
    if (C < 1 || C > 4) return RS_ERR_INVALID_ARG;
    const rs_layout in = rs_layout_hwc(1, H, W, C);
    const rs_layout out = rs_layout_hwc(1, Ho, Wo, C);
    return rs_resize_ex(src, &in, dst, &out, dtype, method, nullptr, stream);
}

rs_status rs_debug_fault(void* stream, uint32_t* code)
{
    if (!code) return RS_ERR_INVALID_ARG;
    unsigned int c = 0;
    rs_status s = cuda_status(read_fault(static_cast<cudaStream_t>(stream), &c));
    *code = c;
    return s;
}

}  // extern "C"
