// Fused serving pre-process on the register-window kernels: a uint8
// interleaved source resampled (bilinear / bicubic, Eqs. 1-5), each
// channel normalised (x - mean) / std in FP32 and stored into its own plane
// as FP16, BF16 or FP32, in one pass (win_body / win_body_x2 with the
// normalising store). One block per (strip, band of output rows, image).
#include <algorithm>
#include <climits>

#include "capi_internal.h"
#include "win_body.cuh"

// Compiled twice so both kernel sets build in parallel: WIN_NORM_PART 0
// (the general form, plus the launch), 1 (the exact-x2 form;
// win_norm_x2.cu).
#ifndef WIN_NORM_PART
#define WIN_NORM_PART 0
#endif

namespace rs {

template <int KT, int C, typename TO, bool X2>
__global__ void __launch_bounds__(kWinThreads, X2 ? 4 : 2)
k_win_norm(const Geom g, const uint8_t* __restrict__ src, TO* __restrict__ dst, const WinCfg cfg, const NormOut no,
           unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int img = blockIdx.z;
    if constexpr (X2)
        win_body_x2<KT, C, uint8_t, TO, true>(g, src + g.sp.offset(img), dst + g.dp.offset(img), cfg, blockIdx.x,
                                              blockIdx.y, sm, fault, no);
    else
        win_body<KT, C, uint8_t, TO, true>(g, src + g.sp.offset(img), dst + g.dp.offset(img), cfg, blockIdx.x,
                                           blockIdx.y, sm, fault, no);
}

static constexpr bool kNormX2 = WIN_NORM_PART == 1;

template <int KT, int C, typename TO>
static void* norm_func() { return reinterpret_cast<void*>(&k_win_norm<KT, C, TO, kNormX2>); }

template <int KT, typename TO>
static void* norm_func_c(int C)
{
    switch (C) {
    case 1: return norm_func<KT, 1, TO>();
    case 2: return norm_func<KT, 2, TO>();
    case 3: return norm_func<KT, 3, TO>();
    default: return norm_func<KT, 4, TO>();
    }
}

static void* norm_kernel_part(int method, int out_dtype, int C)
{
    if (out_dtype == DT_F16) return method == M_BILINEAR ? norm_func_c<2, __half>(C) : norm_func_c<4, __half>(C);
    if (out_dtype == DT_BF16)
        return method == M_BILINEAR ? norm_func_c<2, __nv_bfloat16>(C) : norm_func_c<4, __nv_bfloat16>(C);
    return method == M_BILINEAR ? norm_func_c<2, float>(C) : norm_func_c<4, float>(C);
}

#if WIN_NORM_PART == 1
void* win_norm_kernel_x2(int method, int out_dtype, int C) { return norm_kernel_part(method, out_dtype, C); }
#else
void* win_norm_kernel_x2(int method, int out_dtype, int C);   // win_norm_x2.cu

cudaError_t launch_win_norm(const Geom& g, int method, int out_dtype, const void* src, void* dst, WinCfg c,
                            const NormOut& no, cudaStream_t st)
{
    const bool x2 = win_is_x2(g);
    void* func = x2 ? win_norm_kernel_x2(method, out_dtype, g.C) : norm_kernel_part(method, out_dtype, g.C);
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, kWinThreads, c.band_h <= 0 ? &per_sm : nullptr);
    if (e != cudaSuccess) return e;
    const int SP = kWinThreads * win_pixels(g.C, DT_U8, x2);
    const int64_t strips = ((int64_t)g.Wo + SP - 1) / SP;
    if (c.band_h <= 0) {
        const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
        const int waves = c.waves > 0 ? c.waves : 2;
        const int64_t bands = std::max<int64_t>(1, resident * waves / (strips * g.planes));
        c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.Ho + bands - 1) / bands));
    }
    if (x2 && c.band_h % 2) ++c.band_h;   // bands start on even rows (band_cap = min(256, Ho) is even here)
    if (c.band_h > c.band_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)strips, (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, const_cast<NormOut*>(&no), &fw};
    e = cudaLaunchKernel(func, grid, dim3(kWinThreads), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}
#endif

}  // namespace rs
