// Register-window forward kernel for bilinear and bicubic resampling.
//
// A block owns a strip of tile_w = 4 * 256 output elements and a band of
// output rows; thread t owns strip elements 4t .. 4t+3 for the whole band
// and walks down it. Output row i of the band takes source rows
// f(i), ..., f(i) + KT - 1 (its first tap f(i) never decreases with i), so
// the thread keeps the horizontally interpolated values of the last KT
// source rows in registers and advances a source-row position b:
//   - at position b it interpolates source row b + KT - 1 at its four
//     columns (gathering the taps from a staged FP32 copy of that source
//     row in shared memory) into the register window, which then holds rows
//     b .. b + KT - 1;
//   - every output row i with f(i) == b is blended from the window (packed
//     FP32x2 FMAs), rounded and stored.
// The position loop is unrolled KT times so the window rotates by register
// renaming. Source rows are staged in chunks of R rows; the raw 16-byte
// loads of chunk c + 1 are issued before chunk c is processed and converted
// into the other half of a double buffer afterwards, so one barrier per
// chunk suffices. Out-of-image rows and columns take the edge pixel.
#include <algorithm>
#include <type_traits>

#include "capi_internal.h"
#include "rs_common.cuh"

namespace rs {

static constexpr int kPolyThreads = 256;
static constexpr int kPolyElems = 4 * kPolyThreads;   // strip width in elements
static constexpr int kPolyPrefetch = 4;               // 16-byte units per thread
static constexpr int kPolyMaxBand = 1024;             // rows of the row-tap table

__device__ __forceinline__ uint32_t poly_pack_u8x4(float2 a, float2 b)
{
    const float2 M = make_float2(12582912.0f, 12582912.0f);
    const float2 ra = __fadd2_rn(a, M), rb = __fadd2_rn(b, M);
    const int i0 = __float_as_int(ra.x) - 0x4B400000, i1 = __float_as_int(ra.y) - 0x4B400000;
    const int i2 = __float_as_int(rb.x) - 0x4B400000, i3 = __float_as_int(rb.y) - 0x4B400000;
    uint32_t hi, out;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(hi) : "r"(i3), "r"(i2), "r"(0u));
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(out) : "r"(i1), "r"(i0), "r"(hi));
    return out;
}

template <typename T>
__device__ __forceinline__ void poly_store4(T* p, float2 a, float2 b, int cnt)
{
    if (cnt == 4) {
        if constexpr (sizeof(T) == 1) {
            if ((reinterpret_cast<uintptr_t>(p) & 3) == 0) {
                *reinterpret_cast<uint32_t*>(p) = poly_pack_u8x4(a, b);
                return;
            }
        } else if constexpr (sizeof(T) == 2) {
            if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
                uint2 w;
                if constexpr (std::is_same<T, __half>::value) {
                    __half2 h0 = __float22half2_rn(a), h1 = __float22half2_rn(b);
                    w.x = *reinterpret_cast<uint32_t*>(&h0);
                    w.y = *reinterpret_cast<uint32_t*>(&h1);
                } else {
                    __nv_bfloat162 h0 = __float22bfloat162_rn(a), h1 = __float22bfloat162_rn(b);
                    w.x = *reinterpret_cast<uint32_t*>(&h0);
                    w.y = *reinterpret_cast<uint32_t*>(&h1);
                }
                *reinterpret_cast<uint2*>(p) = w;
                return;
            }
        } else {
            if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
                *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
                return;
            }
        }
    }
    const float v[4] = {a.x, a.y, b.x, b.y};
    #pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < cnt) Store<T>::put(p + k, v[k]);
}

template <typename T>
__device__ __forceinline__ void poly_unpack16(const uint4& u, float* dst)
{
    if constexpr (sizeof(T) == 1) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
        const float2 M = make_float2(-8388608.0f, -8388608.0f);
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 lo = make_float2(__int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7650)),
                                          __int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7651)));
            const float2 hi = make_float2(__int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7652)),
                                          __int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7653)));
            const float2 a = __fadd2_rn(lo, M), b = __fadd2_rn(hi, M);
            *reinterpret_cast<float4*>(dst + 4 * k) = make_float4(a.x, a.y, b.x, b.y);
        }
    } else if constexpr (sizeof(T) == 2) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
        float f[8];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 v;
            if constexpr (std::is_same<T, __half>::value)
                v = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            else
                v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
            f[2 * k] = v.x;
            f[2 * k + 1] = v.y;
        }
        *reinterpret_cast<float4*>(dst) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(dst + 4) = make_float4(f[4], f[5], f[6], f[7]);
    } else {
        *reinterpret_cast<float4*>(dst) = make_float4(__uint_as_float(u.x), __uint_as_float(u.y),
                                                      __uint_as_float(u.z), __uint_as_float(u.w));
    }
}

template <int KT, int C, typename T>
__global__ void __launch_bounds__(kPolyThreads)
k_poly(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const PolyCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;
    const T* s = src + g.sp.offset(plane);
    T* d = dst + g.dp.offset(plane);

    const int64_t WoC = (int64_t)g.Wo * C;
    const int64_t e0 = (int64_t)blockIdx.x * kPolyElems;
    const int nE = (int)min((int64_t)kPolyElems, WoC - e0);
    const int yb = blockIdx.y * cfg.band_h;
    const int ye = min(g.Ho, yb + cfg.band_h);
    const int nrows = ye - yb;

    // Staged columns (as in the streaming kernel): source pixels
    // [px_lo, px_hi] unclamped; position p of a staged row holds element
    // base + p; in-image elements arrive in units of EPU elements from a0,
    // out-of-image columns hold the edge pixel.
    const int j_first = (int)(e0 / C), j_last = (int)((e0 + nE - 1) / C);
    const int px_lo = first_tap<KT>(j_first, g.W, g.Wo, g.coord);
    const int px_hi = first_tap<KT>(j_last, g.W, g.Wo, g.coord) + KT - 1;
    const int EPU = cfg.vec ? 16 / (int)sizeof(T) : 1;
    const int in_lo = max(px_lo, 0) * C, in_hi = (min(px_hi, g.W - 1) + 1) * C;
    const int a0 = (in_lo / EPU) * EPU;
    const int units = (in_hi - a0 + EPU - 1) / EPU;
    const int base = a0 - ((max(0, a0 - px_lo * C) + 3) & ~3);
    const int lpad = max(0, -px_lo) * C;
    const int rpad = max(0, px_hi - (g.W - 1)) * C;
    const int span = max(a0 + units * EPU, (px_hi + 1) * C) - base;
    const int u0 = a0 - base;
    if (span > cfg.swe_max || (u0 & 3) || (cfg.swe_max & 3) || nrows > cfg.band_cap) {   // uniform
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    const int R = cfg.chunk;                               // source rows per chunk
    float* SR = sm;                                        // [2][R][swe_max]
    float* RW = SR + 2 * R * cfg.swe_max;                  // [band_cap][KT]
    int* RF = reinterpret_cast<int*>(RW + cfg.band_cap * KT);   // [band_cap] first taps

    // Row taps of the band.
    for (int i = tid; i < nrows; i += kPolyThreads) {
        float w[KT];
        RF[i] = taps<KT>(yb + i, g.H, g.Ho, g.coord, g.a, w);
        #pragma unroll
        for (int p = 0; p < KT; ++p) RW[i * KT + p] = w[p];
    }

    // Column taps of this thread's four elements.
    const bool active = 4 * tid < nE;
    const int cnt = min(4, nE - 4 * tid);
    int off[4];
    float2 w01[KT], w23[KT];
    {
        float wx[4][KT];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int el = 4 * tid + k;
            if (el < nE) {
                const int64_t e = e0 + el;
                const int j = (int)(e / C), c = (int)(e - (int64_t)j * C);
                const int f = taps<KT>(j, g.W, g.Wo, g.coord, g.a, wx[k]);
                off[k] = f * C + c - base;
            } else {
                off[k] = 0;
                #pragma unroll
                for (int q = 0; q < KT; ++q) wx[k][q] = 0.0f;
            }
        }
        #pragma unroll
        for (int q = 0; q < KT; ++q) {
            w01[q] = make_float2(wx[0][q], wx[1][q]);
            w23[q] = make_float2(wx[2][q], wx[3][q]);
        }
    }

    // Staging of source rows r0 .. r0 + nn - 1 (clamped) into SR half h.
    const uint32_t umul = units > 1 ? 0xFFFFFFFFu / (uint32_t)units + 1u : 0u;
    auto split = [&](int u, int& k, int& w) {
        k = units > 1 ? (int)__umulhi((uint32_t)u, umul) : u;
        w = u - k * units;
    };
    auto row_ptr = [&](int r) -> const T* { return s + (int64_t)clampi(r, g.H) * g.src_pitch; };
    auto pads = [&](int r0, int nn, float* dstb) {
        const int npad = lpad + rpad;
        for (int u = tid; u < nn * npad; u += kPolyThreads) {
            const int k = u / npad, p = u - k * npad;
            const int c = p % C;
            const int src_el = p < lpad ? c : (g.W - 1) * C + c;
            const int pos = p < lpad ? (px_lo * C - base) + p : (g.W * C - base) + (p - lpad);
            dstb[k * cfg.swe_max + pos] = Store<T>::load(row_ptr(r0 + k) + src_el);
        }
    };
    uint4 pf[kPolyPrefetch];
    const int pf_cap = kPolyPrefetch * kPolyThreads;
    auto issue = [&](int r0, int nn) {
        #pragma unroll
        for (int i = 0; i < kPolyPrefetch; ++i) {
            const int u = tid + i * kPolyThreads;
            if (u < nn * units) {
                int k, w;
                split(u, k, w);
                pf[i] = __ldg(reinterpret_cast<const uint4*>(row_ptr(r0 + k) + a0 + w * EPU));
            }
        }
    };
    auto commit = [&](int r0, int nn, float* dstb) {
        #pragma unroll
        for (int i = 0; i < kPolyPrefetch; ++i) {
            const int u = tid + i * kPolyThreads;
            if (u < nn * units) {
                int k, w;
                split(u, k, w);
                poly_unpack16<T>(pf[i], dstb + k * cfg.swe_max + u0 + w * EPU);
            }
        }
        if (lpad + rpad) pads(r0, nn, dstb);
    };
    auto stage_sync = [&](int r0, int nn, float* dstb) {
        const int total = nn * units;
        if (cfg.vec) {
            for (int b0 = 0; b0 < total; b0 += pf_cap) {
                #pragma unroll
                for (int i = 0; i < kPolyPrefetch; ++i) {
                    const int u = b0 + tid + i * kPolyThreads;
                    if (u < total) {
                        int k, w;
                        split(u, k, w);
                        pf[i] = __ldg(reinterpret_cast<const uint4*>(row_ptr(r0 + k) + a0 + w * EPU));
                    }
                }
                #pragma unroll
                for (int i = 0; i < kPolyPrefetch; ++i) {
                    const int u = b0 + tid + i * kPolyThreads;
                    if (u < total) {
                        int k, w;
                        split(u, k, w);
                        poly_unpack16<T>(pf[i], dstb + k * cfg.swe_max + u0 + w * EPU);
                    }
                }
            }
        } else {
            for (int b0 = 0; b0 < total; b0 += 4 * kPolyThreads) {
                float v[4];
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = b0 + tid + i * kPolyThreads;
                    if (u < total) {
                        int k, w;
                        split(u, k, w);
                        v[i] = Store<T>::load(row_ptr(r0 + k) + a0 + w);
                    }
                }
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = b0 + tid + i * kPolyThreads;
                    if (u < total) {
                        int k, w;
                        split(u, k, w);
                        dstb[k * cfg.swe_max + u0 + w] = v[i];
                    }
                }
            }
        }
        if (lpad + rpad) pads(r0, nn, dstb);
    };

    // Horizontal interpolation of a staged row at this thread's columns.
    auto hrow = [&](const float* Sr, float2& h01, float2& h23) {
        h01 = make_float2(0.0f, 0.0f);
        h23 = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int q = 0; q < KT; ++q) {
            h01 = __ffma2_rn(w01[q], make_float2(Sr[off[0] + q * C], Sr[off[1] + q * C]), h01);
            h23 = __ffma2_rn(w23[q], make_float2(Sr[off[2] + q * C], Sr[off[3] + q * C]), h23);
        }
    };

    __syncthreads();   // row taps visible
    const int b_first = RF[0];
    const int b_last = RF[nrows - 1];
    // Source rows in order: b_first .. b_last + KT - 1, in chunks of R.
    const int r_first = b_first, r_end = b_last + KT;      // [r_first, r_end)
    int chunk_lo = r_first;
    int nn = min(R, r_end - chunk_lo);
    stage_sync(chunk_lo, nn, SR);
    int next_lo = chunk_lo + nn;
    int next_nn = min(R, r_end - next_lo);
    bool pref = cfg.vec && next_nn > 0 && next_nn * units <= pf_cap;
    __syncthreads();
    if (pref) issue(next_lo, next_nn);
    int half = 0;

    // Register window: h[p] holds source row (b + p) at position b.
    float2 h01[KT], h23[KT];
    int i = 0;                 // next output row of the band
    int b = b_first;           // current position
    // Prime rows b_first .. b_first + KT - 2 (all in the first chunk: R >= KT).
    #pragma unroll
    for (int p = 0; p < KT - 1; ++p) hrow(SR + p * cfg.swe_max, h01[p], h23[p]);
    int r = b_first + KT - 1;  // next source row to interpolate (newest window row)

    // Emit output rows whose first tap is b, from window slots (in order) s[0..KT).
    auto emit = [&](const int* slot) {
        while (i < nrows && RF[i] == b) {
            float2 v01 = make_float2(0.0f, 0.0f), v23 = make_float2(0.0f, 0.0f);
            #pragma unroll
            for (int p = 0; p < KT; ++p) {
                const float wy = RW[i * KT + p];
                const float2 w2 = make_float2(wy, wy);
                v01 = __ffma2_rn(w2, h01[slot[p]], v01);
                v23 = __ffma2_rn(w2, h23[slot[p]], v23);
            }
            if (active) poly_store4<T>(d + (int64_t)(yb + i) * g.dst_pitch + e0 + 4 * tid, v01, v23, cnt);
            ++i;
        }
    };

    while (b <= b_last) {
        #pragma unroll
        for (int u = 0; u < KT; ++u) {
            if (b <= b_last) {
                // Make source row r = b + KT - 1 available in the staged chunk.
                if (r >= chunk_lo + nn) {
                    // Move to the next chunk. The other half held chunk k-1,
                    // whose reads all precede the barrier of the previous
                    // switch, so it can be overwritten now; the barrier below
                    // publishes the new chunk.
                    half ^= 1;
                    float* dstb = SR + half * R * cfg.swe_max;
                    if (pref) commit(next_lo, next_nn, dstb);
                    else stage_sync(next_lo, next_nn, dstb);
                    chunk_lo = next_lo;
                    nn = next_nn;
                    next_lo = chunk_lo + nn;
                    next_nn = min(R, r_end - next_lo);
                    pref = cfg.vec && next_nn > 0 && next_nn * units <= pf_cap;
                    __syncthreads();
                    if (pref) issue(next_lo, next_nn);
                }
                // the newest row goes into slot (u + KT - 1) % KT
                const int ns = (u + KT - 1) % KT;
                hrow(SR + half * R * cfg.swe_max + (r - chunk_lo) * cfg.swe_max, h01[ns], h23[ns]);
                ++r;
                int slot[KT];
                #pragma unroll
                for (int p = 0; p < KT; ++p) slot[p] = (u + p) % KT;
                emit(slot);
                ++b;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side

static int poly_span_bound(int k, int n, int m, int KT)
{
    const int64_t num = (int64_t)(k - 1) * n;
    return (int)((num + m - 1) / m) + KT;
}

bool poly_config(const Geom& g, int method, int dtype, const void* src, PolyCfg& c)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return false;
    const int KT = method_taps(method);
    const int es = (int)dtype_size(dtype);
    if (c.chunk < KT) return false;
    const uintptr_t basep = reinterpret_cast<uintptr_t>(src);
    const bool planar = g.sp.cp > 1 || g.planes > 1;
    c.vec = (basep % 16 == 0) && ((g.src_pitch * es) % 16 == 0) && (((int64_t)g.W * g.C * es) % 16 == 0) &&
            (!planar || ((g.sp.n_stride * es) % 16 == 0 && (g.sp.c_stride * es) % 16 == 0)) ? 1 : 0;
    const int EPU = c.vec ? 16 / es : 1;
    const int kpx = (kPolyElems + g.C - 1) / g.C + 1;
    const int span_px = poly_span_bound(kpx, g.W, g.Wo, KT);
    c.swe_max = ((span_px * g.C + 2 * EPU + 4) + 3) & ~3;
    c.band_cap = std::min(kPolyMaxBand, g.Ho);
    c.smem = sizeof(float) * (2 * (size_t)c.chunk * c.swe_max + (size_t)c.band_cap * KT) +
             sizeof(int) * (size_t)c.band_cap;
    return c.smem <= max_smem_per_block();
}

template <int KT, int C, typename T>
static void* poly_func() { return reinterpret_cast<void*>(&k_poly<KT, C, T>); }

template <int KT, typename T>
static void* poly_func_c(int C)
{
    switch (C) {
    case 1: return poly_func<KT, 1, T>();
    case 2: return poly_func<KT, 2, T>();
    case 3: return poly_func<KT, 3, T>();
    default: return poly_func<KT, 4, T>();
    }
}

template <typename T>
static void* poly_func_m(int method, int C)
{
    return method == M_BILINEAR ? poly_func_c<2, T>(C) : poly_func_c<4, T>(C);
}

static void* poly_kernel(int method, int dtype, int C)
{
    switch (dtype) {
    case DT_U8: return poly_func_m<uint8_t>(method, C);
    case DT_F16: return poly_func_m<__half>(method, C);
    case DT_BF16: return poly_func_m<__nv_bfloat16>(method, C);
    default: return poly_func_m<float>(method, C);
    }
}

cudaError_t launch_poly(const Geom& g, int method, int dtype, const void* src, void* dst, PolyCfg c, cudaStream_t st)
{
    void* func = poly_kernel(method, dtype, g.C);
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
    const int64_t strips = ((int64_t)g.Wo * g.C + kPolyElems - 1) / kPolyElems;
    if (c.band_h <= 0) {
        int per_sm = 1;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, kPolyThreads, c.smem);
        if (e != cudaSuccess) return e;
        const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
        const int waves = c.waves > 0 ? c.waves : 2;
        const int64_t bands = std::max<int64_t>(1, (resident * waves + strips * g.planes - 1) / (strips * g.planes));
        c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.Ho + bands - 1) / bands));
    }
    if (c.band_h > c.band_cap) return cudaErrorInvalidValue;
    dim3 grid((unsigned)strips, (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, &fw};
    e = cudaLaunchKernel(func, grid, dim3(kPolyThreads), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace rs
