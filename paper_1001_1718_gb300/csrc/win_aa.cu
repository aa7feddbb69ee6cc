// Antialiased resampling (RS_FLAG_ANTIALIAS) on the general register-window
// form: win_body with TAP_AA, at most K taps per axis (K = 4 or 8), for
// every storage dtype (k_win_aa) and for the fused pre-process's normalised
// planar output (k_win_aa_norm, uint8 source). The launch shape follows
// the window kernel's (strips x bands x planes, bands sized from occupancy).
#include <algorithm>

#include "capi_internal.h"
#include "win_body.cuh"

// Compiled twice so both kernel sets build in parallel: WIN_AA_PART 0
// (k_win_aa), 1 (k_win_aa_norm; win_aa_norm.cu).
#ifndef WIN_AA_PART
#define WIN_AA_PART 0
#endif

namespace rs {

static void* aa_dispatch_c(int C, void* f1, void* f2, void* f3, void* f4)
{
    return C == 1 ? f1 : C == 2 ? f2 : C == 3 ? f3 : f4;
}

static cudaError_t launch_aa_common(const Geom& g, void* func, int P, const void* src, void* dst, WinCfg c,
                                    const NormOut* no, cudaStream_t st)
{
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, kWinThreads, c.band_h <= 0 ? &per_sm : nullptr);
    if (e != cudaSuccess) return e;
    if (c.strip < 32 || c.strip > kWinThreads * P) return cudaErrorInvalidValue;
    const int64_t strips = ((int64_t)g.Wo + c.strip - 1) / c.strip;
    if (c.band_h <= 0) {
        const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
        const int waves = c.waves > 0 ? c.waves : 2;
        const int64_t bands = std::max<int64_t>(1, resident * waves / (strips * g.planes));
        c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.Ho + bands - 1) / bands));
    }
    if (c.band_h > c.band_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)strips, (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    if (no) {
        void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, const_cast<NormOut*>(no), &fw};
        e = cudaLaunchKernel(func, grid, dim3(kWinThreads), args, c.smem, st);
    } else {
        void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, &fw};
        e = cudaLaunchKernel(func, grid, dim3(kWinThreads), args, c.smem, st);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

#if WIN_AA_PART == 0

template <int K, int C, typename T>
__global__ void __launch_bounds__(kWinThreads, 2)
k_win_aa(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const WinCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    win_body<K, C, T, T, false, TAP_AA>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x,
                                        blockIdx.y, sm, fault);
}

template <int K, typename T>
static void* aa_func(int C)
{
    return aa_dispatch_c(C, (void*)&k_win_aa<K, 1, T>, (void*)&k_win_aa<K, 2, T>, (void*)&k_win_aa<K, 3, T>,
                         (void*)&k_win_aa<K, 4, T>);
}

template <typename T>
static void* aa_func_k(int K, int C) { return K == 4 ? aa_func<4, T>(C) : aa_func<8, T>(C); }

cudaError_t launch_win_aa(const Geom& g, int method, int dtype, const void* src, void* dst, int K, WinCfg c,
                          cudaStream_t st)
{
    (void)method;
    void* func = dtype == DT_U8 ? aa_func_k<uint8_t>(K, g.C) : dtype == DT_F16 ? aa_func_k<__half>(K, g.C)
               : dtype == DT_BF16 ? aa_func_k<__nv_bfloat16>(K, g.C) : aa_func_k<float>(K, g.C);
    const int P0 = win_pixels(g.C, dtype, false);
    return launch_aa_common(g, func, K > 4 ? std::max(2, P0 / 2) : P0, src, dst, c, nullptr, st);
}

#else

template <int K, int C, typename TO>
__global__ void __launch_bounds__(kWinThreads, 2)
k_win_aa_norm(const Geom g, const uint8_t* __restrict__ src, TO* __restrict__ dst, const WinCfg cfg, const NormOut no,
              unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int img = blockIdx.z;
    win_body<K, C, uint8_t, TO, true, TAP_AA>(g, src + g.sp.offset(img), dst + g.dp.offset(img), cfg, blockIdx.x,
                                              blockIdx.y, sm, fault, no);
}

template <int K, typename TO>
static void* aan_func(int C)
{
    return aa_dispatch_c(C, (void*)&k_win_aa_norm<K, 1, TO>, (void*)&k_win_aa_norm<K, 2, TO>,
                         (void*)&k_win_aa_norm<K, 3, TO>, (void*)&k_win_aa_norm<K, 4, TO>);
}

template <typename TO>
static void* aan_func_k(int K, int C) { return K == 4 ? aan_func<4, TO>(C) : aan_func<8, TO>(C); }

cudaError_t launch_win_aa_norm(const Geom& g, int method, int out_dtype, const void* src, void* dst, int K, WinCfg c,
                               const NormOut& no, cudaStream_t st)
{
    (void)method;
    void* func = out_dtype == DT_F16 ? aan_func_k<__half>(K, g.C) : out_dtype == DT_BF16 ? aan_func_k<__nv_bfloat16>(K, g.C)
               : aan_func_k<float>(K, g.C);
    const int P0 = win_pixels(g.C, DT_U8, false);
    return launch_aa_common(g, func, K > 4 ? std::max(2, P0 / 2) : P0, src, dst, c, &no, st);
}

#endif

}  // namespace rs
