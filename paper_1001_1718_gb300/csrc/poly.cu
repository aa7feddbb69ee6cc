// Register-window forward kernel for bilinear and bicubic resampling: one
// block per (strip of 1024 output elements, band of output rows, plane);
// the block's work is poly_body (poly_body.cuh).
#include <algorithm>
#include <climits>

#include "capi_internal.h"
#include "poly_body.cuh"

// This file is compiled three times: as poly.cu (POLY_MODE 1, aligned
// staging, plus the host configuration and launch), through poly_shifted.cu
// (POLY_MODE 2, shifted staging) and through poly_x2.cu (POLY_MODE 1 with
// POLY_FIX 2: exactly two output rows per source position), so the three
// sets of kernels build in parallel.
#ifndef POLY_MODE
#define POLY_MODE 1
#endif
#ifndef POLY_FIX
#define POLY_FIX 0
#endif

namespace rs {

template <int KT, int C, typename T, int MODE, int FIX>
__global__ void __launch_bounds__(kPolyThreads, 3)
k_poly(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const PolyCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    poly_body<KT, C, T, MODE, FIX>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x, blockIdx.y,
                              sm, fault);
}

// ---------------------------------------------------------------------------
// Host side

#if POLY_MODE == 1 && POLY_FIX == 0
bool poly_config(const Geom& g, int method, int dtype, const void* src, PolyCfg& c, bool shifted_only)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return false;
    const int KT = method_taps(method);
    const int es = (int)dtype_size(dtype);
    if (c.chunk < KT || c.chunk % KT) return false;   // chunks hold whole groups of KT positions
    const uintptr_t basep = reinterpret_cast<uintptr_t>(src);
    const bool planar = g.sp.cp > 1 || g.planes > 1;
    // 16-byte-aligned rows of whole units (1), else the shifted copies (2).
    c.vec = (basep % 16 == 0) && ((g.src_pitch * es) % 16 == 0) && (((int64_t)g.W * g.C * es) % 16 == 0) &&
            (!planar || ((g.sp.n_stride * es) % 16 == 0 && (g.sp.c_stride * es) % 16 == 0)) && !shifted_only ? 1 : 2;
    const int EPU = c.vec ? 16 / es : 1;
    const int kpx = (kPolyElems + g.C - 1) / g.C + 1;
    const int span_px = tap_span_bound(kpx, g.W, g.Wo, KT, g.coord);
    c.swe_max = ((span_px * g.C + 2 * EPU + 4) + 3) & ~3;
    c.band_cap = std::min(kPolyMaxBand, g.Ho);
    if ((int64_t)c.band_cap * g.dst_pitch >= (int64_t)INT32_MAX) return false;   // 32-bit row offsets
    c.pos_cap = tap_span_bound(c.band_cap, g.H, g.Ho, KT, g.coord);   // source positions of a band
    const size_t tables = sizeof(float) * (2 * (size_t)c.chunk * c.swe_max + (size_t)c.band_cap * KT) +
                          sizeof(int) * ((size_t)c.band_cap + (size_t)c.pos_cap);
    c.raw_off = (int)((tables + 15) & ~(size_t)15);
    c.raw_row = c.vec ? (c.swe_max / EPU + (c.vec == 2 ? 3 : 2)) * 16 : 0;
    c.smem = (size_t)c.raw_off + 3 * (size_t)c.chunk * c.raw_row;
    return c.smem <= max_smem_per_block();
}

#endif

template <int KT, int C, typename T>
static void* poly_func(int) { return reinterpret_cast<void*>(&k_poly<KT, C, T, POLY_MODE, POLY_FIX>); }

template <int KT, typename T>
static void* poly_func_c(int C, int mode)
{
    switch (C) {
    case 1: return poly_func<KT, 1, T>(mode);
    case 2: return poly_func<KT, 2, T>(mode);
    case 3: return poly_func<KT, 3, T>(mode);
    default: return poly_func<KT, 4, T>(mode);
    }
}

template <typename T>
static void* poly_func_m(int method, int C, int mode)
{
    return method == M_BILINEAR ? poly_func_c<2, T>(C, mode) : poly_func_c<4, T>(C, mode);
}

#if POLY_MODE == 1 && POLY_FIX == 0
void* poly_kernel_shifted(int method, int dtype, int C);   // poly_shifted.cu
void* poly_kernel_x2(int method, int dtype, int C);        // poly_x2.cu
static void* poly_kernel(int method, int dtype, int C, int mode)
{
    if (mode == 2) return poly_kernel_shifted(method, dtype, C);
    switch (dtype) {
    case DT_U8: return poly_func_m<uint8_t>(method, C, mode);
    case DT_F16: return poly_func_m<__half>(method, C, mode);
    case DT_BF16: return poly_func_m<__nv_bfloat16>(method, C, mode);
    default: return poly_func_m<float>(method, C, mode);
    }
}
#elif POLY_MODE == 2
void* poly_kernel_shifted(int method, int dtype, int C)
{
    switch (dtype) {
    case DT_U8: return poly_func_m<uint8_t>(method, C, 2);
    case DT_F16: return poly_func_m<__half>(method, C, 2);
    case DT_BF16: return poly_func_m<__nv_bfloat16>(method, C, 2);
    default: return poly_func_m<float>(method, C, 2);
    }
}
#else
void* poly_kernel_x2(int method, int dtype, int C)
{
    switch (dtype) {
    case DT_U8: return poly_func_m<uint8_t>(method, C, 1);
    case DT_F16: return poly_func_m<__half>(method, C, 1);
    case DT_BF16: return poly_func_m<__nv_bfloat16>(method, C, 1);
    default: return poly_func_m<float>(method, C, 1);
    }
}
#endif

#if POLY_MODE == 1 && POLY_FIX == 0

cudaError_t launch_poly(const Geom& g, int method, int dtype, const void* src, void* dst, PolyCfg c, cudaStream_t st)
{
    // The asymmetric map at exactly x2 vertically puts two output rows on
    // every source position; bands of an even number of rows then start on
    // an even row (the last band too: Ho is even), which the x2 kernels need.
    const bool x2 = c.vec == 1 && g.coord == COORD_ASYMMETRIC && (int64_t)g.Ho == 2 * (int64_t)g.H &&
                    (c.band_h <= 0 || c.band_h % 2 == 0);
    void* func = x2 ? poly_kernel_x2(method, dtype, g.C) : poly_kernel(method, dtype, g.C, c.vec);
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, kPolyThreads, c.band_h <= 0 ? &per_sm : nullptr);
    if (e != cudaSuccess) return e;
    const int64_t strips = ((int64_t)g.Wo * g.C + kPolyElems - 1) / kPolyElems;
    if (c.band_h <= 0) {
        const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
        const int waves = c.waves > 0 ? c.waves : 2;
        const int64_t bands = std::max<int64_t>(1, (resident * waves + strips * g.planes - 1) / (strips * g.planes));
        c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.Ho + bands - 1) / bands));
        if (x2 && c.band_h % 2) ++c.band_h;   // band_cap = min(256, Ho) is even here
    }
    if (c.band_h > c.band_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)strips, (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, &fw};
    e = cudaLaunchKernel(func, grid, dim3(kPolyThreads), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

#endif

}  // namespace rs
