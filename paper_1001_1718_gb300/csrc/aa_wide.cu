// Antialiased resampling with more taps per axis than the register-window
// forms hold: the single-image kernels of the vertical-first streaming form
// (aa_vs.cuh, vertical downscales) and of the tiled form (aa_wide.cuh, any
// ratio), for every storage dtype and for the fused pre-process's
// normalised planar output, and their host configuration.
#include <algorithm>
#include <vector>

#include "capi_internal.h"
#include "aa_wide.cuh"
#include "aa_vs.cuh"

namespace rs {

template <int C, typename T, typename TO, bool NORM>
__global__ void __launch_bounds__(kAwNT)
k_aa_wide(const Geom g, const T* __restrict__ src, TO* __restrict__ dst, const AaWideCfg cfg, const NormOut no,
          unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    aa_wide_body<C, T, TO, NORM>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x, blockIdx.y,
                                 sm, fault, no);
}

template <int C, typename T, typename TO, bool NORM, int NA>
__global__ void __launch_bounds__(kVsNT, 3)
k_aa_vs(const Geom g, const T* __restrict__ src, TO* __restrict__ dst, const AaVsCfg cfg, const NormOut no,
        unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    aa_vs_body<C, T, TO, NORM, NA>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x, blockIdx.y,
                                   sm, fault, no);
}

// Largest count and widest span of the antialias taps over the tiles of
// `tile` consecutive outputs along one axis.
static void aa_axis_bounds(int n, int m, int method, int tile, int& kmax, int& span)
{
    kmax = 1;
    span = 1;
    for (int j0 = 0; j0 < m; j0 += tile) {
        const int j1 = std::min(m, j0 + tile) - 1;
        int lo0, hi0, lo1, hi1;
        aa_range(j0, n, m, method, lo0, hi0);
        aa_range(j1, n, m, method, lo1, hi1);
        span = std::max(span, hi1 - lo0);
        for (int j = j0; j <= j1; ++j) {
            int lo, hi;
            aa_range(j, n, m, method, lo, hi);
            kmax = std::max(kmax, hi - lo);
        }
    }
}

bool aa_wide_config(const Geom& g, int method, AaWideCfg& c)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return false;
    if (g.C < 1 || g.C > 4) return false;
    c.method = method;
    int fw = 0;
    aa_axis_bounds(g.W, g.Wo, method, kAwTW, c.KX, fw);
    c.fw = fw;
    for (int TH = 32; TH >= 1; TH /= 2) {
        int KY = 0, nr = 0;
        aa_axis_bounds(g.H, g.Ho, method, TH, KY, nr);
        for (int RG = 8; RG >= 1; RG /= 2) {
            c.TH = TH;
            c.KY = KY;
            c.nr = nr;
            c.RG = RG;
            const size_t tabs = sizeof(float) * ((size_t)kAwTW * c.KX + (size_t)TH * KY) +
                                sizeof(int) * (2 * (size_t)kAwTW + 2 * (size_t)TH);
            c.s_off = (int)((tabs + 15) / 16 * 4);   // in floats, 16-byte aligned
            c.smem = sizeof(float) * ((size_t)c.s_off + (size_t)RG * fw * g.C + (size_t)nr * kAwTW * g.C);
            if (c.smem <= max_smem_per_block()) return true;
        }
    }
    return false;
}

// The vertical-first form: output rows no more than source rows; NA = 4, 6
// or 8 register slots, the fewest with every slot's next row starting at or
// below the previous row's last tap; the widest power-of-two tile (up to 256
// columns) whose footprint fits 4 elements per thread; copy-ring chunks of 8
// rows (4, 2 for wide FP32 rows); bands of the tallest TH (64 .. 8 rows)
// that still gives at least 4 blocks per SM in all and fits ~75 KB of
// shared memory, else the shortest that fits the per-block limit.
bool aa_vs_config(const Geom& g, int method, int dtype, AaVsCfg& c)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return false;
    if (g.C < 1 || g.C > 4 || g.Ho > g.H) return false;
    const int es = (int)dtype_size(dtype);
    c.method = method;
    std::vector<int> lo(g.Ho), hi(g.Ho);
    for (int i = 0; i < g.Ho; ++i) aa_range(i, g.H, g.Ho, method, lo[i], hi[i]);
    c.NA = 0;
    for (int na : {4, 6, 8}) {
        bool ok = true;
        for (int i = 0; i + na < g.Ho && ok; ++i) ok = lo[i + na] >= hi[i];
        if (ok) {
            c.NA = na;
            break;
        }
    }
    if (!c.NA) return false;
    c.TW = 0;
    int span = 0;
    for (int tw = 256; tw >= 8 && !c.TW; tw /= 2) {
        int kx = 0;
        aa_axis_bounds(g.W, g.Wo, method, tw, kx, span);
        if ((int64_t)span * g.C <= (int64_t)kVsNT * kVsE) {
            c.TW = tw;
            c.KX = kx;
        }
    }
    if (!c.TW) return false;
    c.ve = (span * g.C + 3) & ~3;
    c.raw_row = ((span * g.C * es + 15) / 16 + 2) * 16;   // a spare block past the copied ones
    c.chunk = 8;
    while (c.chunk > 2 && (size_t)3 * c.chunk * c.raw_row > 40 * 1024) c.chunk /= 2;
    const int64_t tiles_x = (g.Wo + c.TW - 1) / c.TW;
    bool any = false;
    AaVsCfg fit = c;
    for (int th = 64; th >= 8; th /= 2) {
        int ky = 0, nr = 0;
        aa_axis_bounds(g.H, g.Ho, method, th, ky, nr);
        AaVsCfg t = c;
        t.TH = th;
        t.nr = nr;
        t.smem = (size_t)3 * t.chunk * t.raw_row +
                 sizeof(float) * (kVsNB * (size_t)t.ve + (size_t)t.TW * t.KX + (size_t)nr * t.NA) +
                 sizeof(int) * (2 * (size_t)t.TW + 2 * (size_t)nr);
        if (t.smem > max_smem_per_block()) continue;
        fit = t;
        any = true;
        const int64_t blocks = tiles_x * ((g.Ho + th - 1) / th) * g.planes;
        if (t.smem <= 75 * 1024 && blocks >= 4LL * num_sms()) break;
    }
    if (any) c = fit;
    return any;
}

template <typename T, typename TO, bool NORM, int NA>
static void* aa_vs_func(int C)
{
    return C == 1 ? (void*)&k_aa_vs<1, T, TO, NORM, NA> : C == 2 ? (void*)&k_aa_vs<2, T, TO, NORM, NA>
         : C == 3 ? (void*)&k_aa_vs<3, T, TO, NORM, NA> : (void*)&k_aa_vs<4, T, TO, NORM, NA>;
}

template <typename T, typename TO, bool NORM>
static void* aa_vs_func_na(int NA, int C)
{
    return NA == 4 ? aa_vs_func<T, TO, NORM, 4>(C) : NA == 6 ? aa_vs_func<T, TO, NORM, 6>(C)
                   : aa_vs_func<T, TO, NORM, 8>(C);
}

static cudaError_t launch_aa_vs_common(const Geom& g, void* func, const void* src, void* dst, const AaVsCfg& c,
                                       const NormOut& no, cudaStream_t st)
{
    cudaError_t e = prepare_kernel(func, c.smem, kVsNT, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.Wo + c.TW - 1) / c.TW), (unsigned)((g.Ho + c.TH - 1) / c.TH), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, const_cast<AaVsCfg*>(&c),
                    const_cast<NormOut*>(&no), &fw};
    e = cudaLaunchKernel(func, grid, dim3(kVsNT), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_aa_vs(const Geom& g, int dtype, const void* src, void* dst, const AaVsCfg& c, cudaStream_t st)
{
    void* func = dtype == DT_U8 ? aa_vs_func_na<uint8_t, uint8_t, false>(c.NA, g.C)
               : dtype == DT_F16 ? aa_vs_func_na<__half, __half, false>(c.NA, g.C)
               : dtype == DT_BF16 ? aa_vs_func_na<__nv_bfloat16, __nv_bfloat16, false>(c.NA, g.C)
               : aa_vs_func_na<float, float, false>(c.NA, g.C);
    return launch_aa_vs_common(g, func, src, dst, c, NormOut{}, st);
}

cudaError_t launch_aa_vs_norm(const Geom& g, int out_dtype, const void* src, void* dst, const AaVsCfg& c,
                              const NormOut& no, cudaStream_t st)
{
    void* func = out_dtype == DT_F16 ? aa_vs_func_na<uint8_t, __half, true>(c.NA, g.C)
               : out_dtype == DT_BF16 ? aa_vs_func_na<uint8_t, __nv_bfloat16, true>(c.NA, g.C)
               : aa_vs_func_na<uint8_t, float, true>(c.NA, g.C);
    return launch_aa_vs_common(g, func, src, dst, c, no, st);
}

template <typename T, typename TO, bool NORM>
static void* aa_wide_func(int C)
{
    return C == 1 ? (void*)&k_aa_wide<1, T, TO, NORM> : C == 2 ? (void*)&k_aa_wide<2, T, TO, NORM>
         : C == 3 ? (void*)&k_aa_wide<3, T, TO, NORM> : (void*)&k_aa_wide<4, T, TO, NORM>;
}

static cudaError_t launch_aa_wide_common(const Geom& g, void* func, const void* src, void* dst, const AaWideCfg& c,
                                         const NormOut& no, cudaStream_t st)
{
    cudaError_t e = prepare_kernel(func, c.smem, kAwNT, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.Wo + kAwTW - 1) / kAwTW), (unsigned)((g.Ho + c.TH - 1) / c.TH), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, const_cast<AaWideCfg*>(&c),
                    const_cast<NormOut*>(&no), &fw};
    e = cudaLaunchKernel(func, grid, dim3(kAwNT), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_aa_wide(const Geom& g, int dtype, const void* src, void* dst, const AaWideCfg& c, cudaStream_t st)
{
    void* func = dtype == DT_U8 ? aa_wide_func<uint8_t, uint8_t, false>(g.C)
               : dtype == DT_F16 ? aa_wide_func<__half, __half, false>(g.C)
               : dtype == DT_BF16 ? aa_wide_func<__nv_bfloat16, __nv_bfloat16, false>(g.C)
               : aa_wide_func<float, float, false>(g.C);
    return launch_aa_wide_common(g, func, src, dst, c, NormOut{}, st);
}

cudaError_t launch_aa_wide_norm(const Geom& g, int out_dtype, const void* src, void* dst, const AaWideCfg& c,
                                const NormOut& no, cudaStream_t st)
{
    void* func = out_dtype == DT_F16 ? aa_wide_func<uint8_t, __half, true>(g.C)
               : out_dtype == DT_BF16 ? aa_wide_func<uint8_t, __nv_bfloat16, true>(g.C)
               : aa_wide_func<uint8_t, float, true>(g.C);
    return launch_aa_wide_common(g, func, src, dst, c, no, st);
}

}  // namespace rs
