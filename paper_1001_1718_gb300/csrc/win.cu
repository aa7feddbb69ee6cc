// Register-window forward kernel for bilinear and bicubic resampling: one
// block per (strip of kWinThreads * P output pixels, band of output rows,
// plane); the block's work is win_body (win_body.cuh).
#include <algorithm>
#include <climits>

#include "capi_internal.h"
#include "win_body.cuh"

// This file is compiled four times so the kernel sets build in parallel:
// WIN_PART 0 (uint8 / FP16, general; plus the host configuration and
// launch), 1 (BF16 / FP32, general), 2 (uint8 / FP16, exact x2) and 3
// (BF16 / FP32, exact x2); win_p1.cu .. win_p3.cu define the part.
#ifndef WIN_PART
#define WIN_PART 0
#endif

namespace rs {

// The general form keeps up to ~144 registers per thread (a 128-register cap
// measured 1.3x slower: values recomputed instead of kept); the exact-x2 form
// fits in 128 with four blocks per SM.
template <int KT, int C, typename T, bool X2>
__global__ void __launch_bounds__(kWinThreads, X2 ? 4 : 2)
k_win(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const WinCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    if constexpr (X2)
        win_body_x2<KT, C, T>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x, blockIdx.y, sm,
                              fault);
    else
        win_body<KT, C, T>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x, blockIdx.y, sm, fault);
}

static constexpr bool kPartX2 = WIN_PART >= 2;

template <int KT, int C, typename T>
static void* win_func() { return reinterpret_cast<void*>(&k_win<KT, C, T, kPartX2>); }

template <int KT, typename T>
static void* win_func_c(int C)
{
    switch (C) {
    case 1: return win_func<KT, 1, T>();
    case 2: return win_func<KT, 2, T>();
    case 3: return win_func<KT, 3, T>();
    default: return win_func<KT, 4, T>();
    }
}

template <typename T>
static void* win_func_m(int method, int C)
{
    return method == M_BILINEAR ? win_func_c<2, T>(C) : win_func_c<4, T>(C);
}

#if WIN_PART == 0
void* win_kernel_x2_lo(int method, int dtype, int C);
void* win_kernel_x2_hi(int method, int dtype, int C);
void* win_kernel_gen_hi(int method, int dtype, int C);

static void* win_kernel(int method, int dtype, int C, bool x2)
{
    const bool lo = dtype == DT_U8 || dtype == DT_F16;
    if (x2) return lo ? win_kernel_x2_lo(method, dtype, C) : win_kernel_x2_hi(method, dtype, C);
    if (!lo) return win_kernel_gen_hi(method, dtype, C);
    return dtype == DT_U8 ? win_func_m<uint8_t>(method, C) : win_func_m<__half>(method, C);
}
#elif WIN_PART == 1
void* win_kernel_gen_hi(int method, int dtype, int C)
{
    return dtype == DT_BF16 ? win_func_m<__nv_bfloat16>(method, C) : win_func_m<float>(method, C);
}
#elif WIN_PART == 2
void* win_kernel_x2_lo(int method, int dtype, int C)
{
    return dtype == DT_U8 ? win_func_m<uint8_t>(method, C) : win_func_m<__half>(method, C);
}
#else
void* win_kernel_x2_hi(int method, int dtype, int C)
{
    return dtype == DT_BF16 ? win_func_m<__nv_bfloat16>(method, C) : win_func_m<float>(method, C);
}
#endif

#if WIN_PART == 0

// ---------------------------------------------------------------------------
// Host side

int win_pixels(int C, int dtype, bool x2)
{
    const int es = (int)dtype_size(dtype);
    if (!x2) return C == 1 ? 8 : C == 4 ? 2 : 4;
    if (C == 1) return es == 4 ? 4 : 8;
    if (C == 2) return es == 4 ? 2 : 4;
    if (C == 3) return es == 1 ? 4 : 2;
    return 2;
}

bool win_is_x2(const Geom& g)
{
    return g.coord == COORD_ASYMMETRIC && (int64_t)g.Wo == 2 * (int64_t)g.W && (int64_t)g.Ho == 2 * (int64_t)g.H;
}

static size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

bool win_config(const Geom& g, int method, int dtype, WinCfg& c, bool allow_x2)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return false;
    if (g.C < 1 || g.C > 4) return false;
    const int KT = method_taps(method);
    if (c.chunk < KT || c.chunk % KT || c.chunk > 32) return false;   // chunks hold whole groups of KT rows
    const int es = (int)dtype_size(dtype);
    const bool x2 = allow_x2 && win_is_x2(g);
    const int P = win_pixels(g.C, dtype, x2);
    const int SP = kWinThreads * P;
    // source pixels a strip's footprint can span
    const int span_px = tap_span_bound(SP, g.W, g.Wo, KT, g.coord);
    const int per = (span_px * g.C * es + 15) / 16 + 1;   // raw 16-byte blocks per row
    if (x2) {
        // raw rows only (three slots), long enough for every thread's footprint words
        const int half = P / 2 * g.C;
        const int fpl = (P / 2 + KT - 1) * g.C;
        const int nf = (fpl * es + 3) / 4, nr = es == 4 ? nf : nf + 1;
        const int need = std::max(per * 16, 16 + (kWinThreads - 1) * half * es + 4 * nr);
        c.swe = 0;
        c.raw_row = (need + 15) & ~15;
    } else {    // channel-planar FP32 rows and a two-slot raw ring
        c.swe = g.C * ((span_px + 3) & ~3);
        c.raw_row = per * 16;
    }
    c.band_cap = std::min(kWinMaxBand, g.Ho);
    if ((int64_t)c.band_cap * g.dst_pitch >= (int64_t)INT32_MAX) return false;   // 32-bit row offsets
    c.pos_cap = tap_span_bound(c.band_cap, g.H, g.Ho, KT, g.coord);
    if (x2) {
        c.tab_off = c.raw_off = 0;
        c.smem = 3 * (size_t)c.chunk * c.raw_row;
    } else {
        c.tab_off = (int)align16(sizeof(float) * (size_t)c.chunk * c.swe);
        const size_t tabs = sizeof(float2) * (size_t)c.band_cap * KT + sizeof(int) * ((size_t)c.band_cap + c.pos_cap);
        c.raw_off = (int)align16((size_t)c.tab_off + tabs);
        c.smem = (size_t)c.raw_off + 2 * (size_t)c.chunk * c.raw_row;
    }
    return c.smem <= max_smem_per_block();
}

// The most antialias taps an output has on axis n -> m (the integer bounds
// the kernels use).
static int aa_axis_taps(int n, int m, int method)
{
    int k = 0;
    for (int j = 0; j < m; ++j) {
        int lo, hi;
        aa_range(j, n, m, method, lo, hi);
        k = std::max(k, hi - lo);
    }
    return k;
}

int antialias_taps(const Geom& g, int method)
{
    return std::max(aa_axis_taps(g.H, g.Ho, method), aa_axis_taps(g.W, g.Wo, method));
}

bool win_config_aa(const Geom& g, int method, int dtype, int K, WinCfg& c)
{
    if ((method != M_BILINEAR && method != M_BICUBIC) || (K != 4 && K != 8)) return false;
    if (g.C < 1 || g.C > 4) return false;
    if (c.chunk < K || c.chunk % K || c.chunk > 32) return false;
    const int es = (int)dtype_size(dtype);
    const int P0 = win_pixels(g.C, dtype, false);
    const int P = K > 4 ? std::max(2, P0 / 2) : P0;
    const int SP = kWinThreads * P;
    c.band_cap = std::min(kWinMaxBand, g.Ho);
    if ((int64_t)c.band_cap * g.dst_pitch >= (int64_t)INT32_MAX) return false;
    c.pos_cap = (int)(((int64_t)(c.band_cap - 1) * g.H + g.Ho - 1) / g.Ho) + 2;
    c.aa_method = method;
    // The widest strip (128 P pixels, halved down to one warp's 32) whose
    // footprint fits in shared memory.
    for (int strip = std::min(SP, std::max(32, (g.Wo + 31) & ~31)); strip >= 32; strip /= 2) {
        // first taps advance by at most ceil(n / m) + 1 per output
        const int span_px = (int)(((int64_t)(strip - 1) * g.W + g.Wo - 1) / g.Wo) + 1 + K;
        const int per = (span_px * g.C * es + 15) / 16 + 1;
        c.strip = strip;
        c.swe = g.C * ((span_px + 3) & ~3);
        c.raw_row = per * 16;
        c.tab_off = (int)align16(sizeof(float) * (size_t)c.chunk * c.swe);
        const size_t tabs = sizeof(float2) * (size_t)c.band_cap * K + sizeof(int) * ((size_t)c.band_cap + c.pos_cap);
        c.raw_off = (int)align16((size_t)c.tab_off + tabs);
        c.smem = (size_t)c.raw_off + 2 * (size_t)c.chunk * c.raw_row;
        if (c.smem <= max_smem_per_block()) return true;
    }
    return false;
}

cudaError_t launch_win(const Geom& g, int method, int dtype, const void* src, void* dst, WinCfg c, cudaStream_t st)
{
    const bool x2 = win_is_x2(g);
    void* func = win_kernel(method, dtype, g.C, x2);
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, kWinThreads, c.band_h <= 0 ? &per_sm : nullptr);
    if (e != cudaSuccess) return e;
    const int SP = kWinThreads * win_pixels(g.C, dtype, x2);
    const int64_t strips = ((int64_t)g.Wo + SP - 1) / SP;
    if (c.band_h <= 0) {
        const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
        // two blocks per resident slot; one for a single plane's vertical
        // downscale, whose bands stage several source rows per output row
        // (fewer, longer bands measured faster there)
        const int waves = c.waves > 0 ? c.waves : g.Ho < g.H && g.planes == 1 ? 1 : 2;
        // at most `waves` blocks per resident slot: a partial extra wave would run alone
        const int64_t bands = std::max<int64_t>(1, resident * waves / (strips * g.planes));
        c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.Ho + bands - 1) / bands));
    }
    if (x2 && c.band_h % 2) ++c.band_h;   // bands start on even rows (band_cap = min(256, Ho) is even here)
    if (c.band_h > c.band_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)strips, (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, &fw};
    e = cudaLaunchKernel(func, grid, dim3(kWinThreads), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

#endif

}  // namespace rs
