// Device building blocks shared by the resampling kernels: the exact integer
// coordinate map (Eqs. 1-4), per-method tap weights in FP32, and storage
// conversions. Nothing here allocates or touches global state.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rs_internal.h"

namespace rs {

// ---------------------------------------------------------------------------
// Coordinate map.
//
// Output index j of an axis of m outputs over n source samples maps to the
// rational source coordinate x = num / den (Eq. 1 with scale = m / n):
//   asymmetric:    num = j n,            den = m
//   half-pixel:    num = (2j + 1) n - m, den = 2 m
//   align-corners: num = j (n - 1),      den = m - 1  (num = 0, den = 1 if m = 1)
// i0 = floor(x) and t = (num - i0 den) / den (Eqs. 2-4). The quotient is
// estimated in FP32 (error < 1 for |num| < 2^34 and den <= 2^17) and then
// corrected in exact 64-bit integer arithmetic, so i0 is exact and t takes a
// single rounding (the remainder and den are exact FP32 integers).
// ---------------------------------------------------------------------------

__device__ __forceinline__ int floor_div_exact(int64_t num, int64_t den, int64_t& rem)
{
    int64_t q = (int64_t)floorf((float)num / (float)den);
    int64_t r = num - q * den;
    if (r < 0) { q -= 1; r += den; }
    else if (r >= den) { q += 1; r -= den; }
    rem = r;
    return (int)q;
}

__device__ __forceinline__ void axis_map(int j, int n, int m, int coord, int& i0, float& t)
{
    int64_t num, den;
    if (coord == COORD_ASYMMETRIC) { num = (int64_t)j * n; den = m; }
    else if (coord == COORD_HALF_PIXEL) { num = (int64_t)(2 * j + 1) * n - m; den = 2 * (int64_t)m; }
    else if (m > 1) { num = (int64_t)j * (n - 1); den = m - 1; }
    else { num = 0; den = 1; }
    int64_t rem;
    i0 = floor_div_exact(num, den, rem);
    t = __fdiv_rn((float)rem, (float)den);
}

// Nearest sample: i0 (asymmetric, Eq. 2's x1) or floor(x + 1/2) (half-pixel,
// align-corners).
__device__ __forceinline__ int nearest_index(int j, int n, int m, int coord)
{
    int64_t rem;
    if (coord == COORD_ASYMMETRIC) return floor_div_exact((int64_t)j * n, m, rem);
    if (coord == COORD_HALF_PIXEL) return floor_div_exact((int64_t)(2 * j + 1) * n, 2 * (int64_t)m, rem);
    if (m <= 1) return 0;
    return floor_div_exact((int64_t)2 * j * (n - 1) + (m - 1), 2 * (int64_t)(m - 1), rem);
}

// Index of the first (unclamped) tap of output j for a KT-tap method:
// nearest -> the nearest sample, bilinear -> i0, bicubic -> i0 - 1.
template <int KT>
__device__ __forceinline__ int first_tap(int j, int n, int m, int coord)
{
    if (KT == 1) return nearest_index(j, n, m, coord);
    int i0; float t;
    axis_map(j, n, m, coord, i0, t);
    return KT == 4 ? i0 - 1 : i0;
}

// Tap weights of fraction t. Keys' kernel with parameter a, written in terms
// of t and s = 1 - t:
//   K(1+t) = a t s^2,  K(t) = 1 - t^2 (1 + (a+2) s),
//   K(1-t) = 1 - s^2 (1 + (a+2) t),  K(2-t) = a s t^2,
// which is exact at t = 0 (weights 0, 1, 0, 0) for every a.
template <int KT>
__device__ __forceinline__ void tap_weights(float t, float a, float* w)
{
    if (KT == 1) { w[0] = 1.0f; return; }
    const float s = 1.0f - t;
    if (KT == 2) { w[0] = s; w[1] = t; return; }
    const float a2 = a + 2.0f;
    w[0] = a * t * s * s;
    w[1] = fmaf(-t * t, fmaf(a2, s, 1.0f), 1.0f);
    w[2] = fmaf(-s * s, fmaf(a2, t, 1.0f), 1.0f);
    w[3] = a * s * t * t;
}

// First tap and weights of output j.
template <int KT>
__device__ __forceinline__ int taps(int j, int n, int m, int coord, float a, float* w)
{
    if (KT == 1) { w[0] = 1.0f; return nearest_index(j, n, m, coord); }
    int i0; float t;
    axis_map(j, n, m, coord, i0, t);
    tap_weights<KT>(t, a, w);
    return KT == 4 ? i0 - 1 : i0;
}

__device__ __forceinline__ int clampi(int i, int n)
{
    return min(max(i, 0), n - 1);
}

// ---------------------------------------------------------------------------
// Storage conversions. Loads widen exactly to FP32. Stores round to nearest
// even; uint8 clamps to [0, 255] first (NaN -> 0): adding 1.5 * 2^23 in
// round-to-nearest-even leaves round(v) in the low mantissa byte.
// ---------------------------------------------------------------------------

template <typename T> struct Store;

template <> struct Store<uint8_t> {
    static __device__ __forceinline__ float load(const uint8_t* p) { return (float)__ldg(p); }
    static __device__ __forceinline__ uint32_t bits(float v)
    {
        v = fminf(fmaxf(v, 0.0f), 255.0f);
        return __float_as_uint(__fadd_rn(v, 12582912.0f)) & 0xFFu;
    }
    static __device__ __forceinline__ void put(uint8_t* p, float v) { *p = (uint8_t)bits(v); }
};

template <> struct Store<__half> {
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void put(__half* p, float v) { *p = __float2half_rn(v); }
};

template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void put(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

template <> struct Store<float> {
    static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void put(float* p, float v) { *p = v; }
};

// Store four consecutive elements (the first `cnt` of them), vectorised when
// all four are in range and the address is aligned to the vector size.
template <typename T>
__device__ __forceinline__ void store4(T* p, const float v[4], int cnt)
{
    if (cnt == 4) {
        if constexpr (sizeof(T) == 1) {
            if ((reinterpret_cast<uintptr_t>(p) & 3) == 0) {
                uint32_t w = Store<uint8_t>::bits(v[0]) | (Store<uint8_t>::bits(v[1]) << 8) |
                             (Store<uint8_t>::bits(v[2]) << 16) | (Store<uint8_t>::bits(v[3]) << 24);
                *reinterpret_cast<uint32_t*>(p) = w;
                return;
            }
        } else if constexpr (sizeof(T) == 2) {
            if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
                T h[4];
                #pragma unroll
                for (int k = 0; k < 4; ++k) Store<T>::put(&h[k], v[k]);
                *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(h);
                return;
            }
        } else {
            if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
                *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
                return;
            }
        }
    }
    #pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < cnt) Store<T>::put(p + k, v[k]);
}

// Fault word: a kernel that detects an internal bound violation records a
// code here (first one wins) and skips the access instead of trapping.
__device__ __forceinline__ void report_fault(unsigned int* fault, unsigned int code)
{
    if (fault) atomicCAS(fault, 0u, code);
}

// Antialias taps of output j of an axis of m outputs over n samples (the
// definition in rs_resize_ex's RS_FLAG_ANTIALIAS): the kernel stretched by
// f = max(n / m, 1), taps cut to [0, n), weights renormalised. In exact
// integer arithmetic with F = max(n, m) = m f: the centre is
// c = (2j + 1) n / (2m), so the taps run from floor(((2j+1) n - 2 R F + m) /
// (2m)) to floor(((2j+1) n + 2 R F + m) / (2m)) - 1, and tap i sits at
// u = ((2i+1) m - (2j+1) n) / (2F) kernel units. (Where that bound is an
// exact integer an FP64 evaluation may add or drop the boundary tap; its
// weight K(+-R) is zero.) The weights are evaluated in FP32.
__host__ __device__ inline int64_t floor_div_i64(int64_t a, int64_t b)   // b > 0
{
    const int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__host__ __device__ inline void aa_range(int j, int n, int m, int method, int& lo, int& hi)
{
    const int64_t R = method == M_BILINEAR ? 1 : 2;
    const int64_t F = n > m ? n : m;
    const int64_t a = (int64_t)(2 * j + 1) * n + m;
    const int64_t l = floor_div_i64(a - 2 * R * F, 2 * (int64_t)m);
    const int64_t h = floor_div_i64(a + 2 * R * F, 2 * (int64_t)m);
    lo = (int)(l < 0 ? 0 : l);
    hi = (int)(h > n ? n : h);   // exclusive
}

// Unnormalised antialias weight of source index i for the output whose
// centre is cj / (2 n) (cj = (2 j + 1) n): the kernel at the stretched
// distance u = |(2 i + 1) m - cj| / (2 max(n, m)).
__device__ __forceinline__ float aa_kernel(int i, int m, int64_t cj, float inv2F, int method, float a)
{
    const float u = fabsf((float)((int64_t)(2 * i + 1) * m - cj) * inv2F);
    if (method == M_BILINEAR) return fmaxf(0.0f, 1.0f - u);
    if (u <= 1.0f) return ((a + 2.0f) * u - (a + 3.0f)) * u * u + 1.0f;
    if (u < 2.0f) return ((a * u - 5.0f * a) * u + 8.0f * a) * u - 4.0f * a;
    return 0.0f;
}

template <int K>
__device__ __forceinline__ void aa_taps(int j, int n, int m, int method, float a, int& lo, float* w,
                                        unsigned int* fault)
{
    int hi;
    aa_range(j, n, m, method, lo, hi);
    int cnt = max(0, hi - lo);
    if (cnt > K) {   // excluded by the host
        report_fault(fault, FAULT_BWD_TAPS);
        cnt = K;
    }
    const float inv2F = 1.0f / (2.0f * (float)max(n, m));
    const int64_t cj = (int64_t)(2 * j + 1) * n;
    float tot = 0.0f;
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = k < cnt ? aa_kernel(lo + k, m, cj, inv2F, method, a) : 0.0f;
        w[k] = v;
        tot += v;
    }
    const float inv = tot != 0.0f ? 1.0f / tot : 1.0f;
    #pragma unroll
    for (int k = 0; k < K; ++k) w[k] *= inv;
}

// The renormalised antialias weight of source index i in output j's taps
// (0 outside them): the value aa_taps gives that tap, for any tap count.
__device__ __forceinline__ float aa_weight(int j, int i, int n, int m, int method, float a)
{
    int lo, hi;
    aa_range(j, n, m, method, lo, hi);
    const float inv2F = 1.0f / (2.0f * (float)max(n, m));
    const int64_t cj = (int64_t)(2 * j + 1) * n;
    float tot = 0.0f, wi = 0.0f;
    for (int t = lo; t < hi; ++t) {
        const float v = aa_kernel(t, m, cj, inv2F, method, a);
        tot += v;
        if (t == i) wi = v;
    }
    return wi * (tot != 0.0f ? 1.0f / tot : 1.0f);
}

// Renormalised antialias taps of output j (any count up to K): w[0, cnt)
// and the first tap lo; cnt is returned.
__device__ __forceinline__ int aa_taps_n(int j, int n, int m, int method, float a, int K, int& lo, float* w,
                                         unsigned int* fault)
{
    int hi;
    aa_range(j, n, m, method, lo, hi);
    int cnt = max(0, hi - lo);
    if (cnt > K) {   // excluded by the host
        report_fault(fault, FAULT_BWD_TAPS);
        cnt = K;
    }
    const float inv2F = 1.0f / (2.0f * (float)max(n, m));
    const int64_t cj = (int64_t)(2 * j + 1) * n;
    float tot = 0.0f;
    for (int k = 0; k < cnt; ++k) {
        const float v = aa_kernel(lo + k, m, cj, inv2F, method, a);
        w[k] = v;
        tot += v;
    }
    const float inv = tot != 0.0f ? 1.0f / tot : 1.0f;
    for (int k = 0; k < cnt; ++k) w[k] *= inv;
    return cnt;
}

// The work of one block: output tile (bx, by) of one plane (s, d: the
// plane's first source / output element). Shared memory: cfg.smem bytes.
}  // namespace rs
