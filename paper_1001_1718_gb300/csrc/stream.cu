// Streaming forward kernel: one block per (column strip, row band) of one
// plane, walking down its band in chunks of output rows.
//
// Per block, once:
//   - each thread computes the column taps of its four output elements
//     (Eqs. 1-4 on the x axis) into registers;
// per chunk of chunk_h output rows:
//   - the chunk's row taps go to a double-buffered table in shared memory;
//   - the source rows the chunk needs and no earlier chunk loaded are staged
//     in shared memory as FP32. With 16-byte-aligned rows these are 16-byte
//     vector loads issued one chunk AHEAD into registers, so the loads of
//     chunk c+1 are in flight while chunk c computes;
//   - horizontal pass: each new source row is interpolated at the strip's
//     output columns once, into a power-of-two ring of rows in shared memory
//     (rows shared by neighbouring chunks are not recomputed);
//   - vertical pass: each output row blends its taps' ring rows (packed
//     FP32x2 FMAs), rounds to the storage type and stores four consecutive
//     elements per thread. Rows whose weights are exactly (0, 1, 0, 0) or
//     (1, 0) copy a ring row.
// Edge replication: every tap index is clamped to the image before it is
// turned into a shared-memory offset, so staged rows hold only real pixels.
#include <algorithm>
#include <type_traits>

#include "capi_internal.h"
#include "rs_common.cuh"

namespace rs {

static constexpr int kThreads = 256;
static constexpr int kPrefetch = 4;     // 16-byte units in flight per thread
static constexpr int kRowBias = 1 << 20; // keeps biased row indices positive
static constexpr int kMaxBand = 512;     // rows of the per-block row-tap table

// uint8 pack of four FP32 values: clamp to [0, 255] and round half to even.
// Adding 1.5 * 2^23 rounds to an integer in the low mantissa bits (round to
// nearest even); the saturating pack clamps each value to 0..255.
__device__ __forceinline__ uint32_t pack_u8x4(float2 a, float2 b)
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
__device__ __forceinline__ void store4v(T* p, float2 a, float2 b, int cnt)
{
    if (cnt == 4) {
        if constexpr (sizeof(T) == 1) {
            if ((reinterpret_cast<uintptr_t>(p) & 3) == 0) {
                *reinterpret_cast<uint32_t*>(p) = pack_u8x4(a, b);
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

// Position of strip element e in a padded ring row (4 floats per 16).
__device__ __forceinline__ int hpos(int e) { return e + ((e >> 4) << 2); }

// Store EV = 16 / sizeof(T) consecutive elements (the first `cnt`) given as
// float pairs: one 16-byte store when all are in range and the address is
// 16-byte aligned, else groups of four.
template <typename T>
__device__ __forceinline__ void store16(T* p, const float2* v, int cnt)
{
    constexpr int EV = 16 / (int)sizeof(T);
    if (cnt == EV && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        uint4 w;
        if constexpr (sizeof(T) == 1) {
            w.x = pack_u8x4(v[0], v[1]);
            w.y = pack_u8x4(v[2], v[3]);
            w.z = pack_u8x4(v[4], v[5]);
            w.w = pack_u8x4(v[6], v[7]);
        } else if constexpr (sizeof(T) == 2) {
            uint32_t h[4];
            #pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (std::is_same<T, __half>::value) {
                    __half2 x = __float22half2_rn(v[k]);
                    h[k] = *reinterpret_cast<uint32_t*>(&x);
                } else {
                    __nv_bfloat162 x = __float22bfloat162_rn(v[k]);
                    h[k] = *reinterpret_cast<uint32_t*>(&x);
                }
            }
            w = make_uint4(h[0], h[1], h[2], h[3]);
        } else {
            w = make_uint4(__float_as_uint(v[0].x), __float_as_uint(v[0].y), __float_as_uint(v[1].x),
                           __float_as_uint(v[1].y));
        }
        *reinterpret_cast<uint4*>(p) = w;
        return;
    }
    #pragma unroll
    for (int gq = 0; gq < EV / 4; ++gq)
        if (cnt > 4 * gq) store4v<T>(p + 4 * gq, v[2 * gq], v[2 * gq + 1], min(4, cnt - 4 * gq));
}

// 16 bytes of storage -> FP32 in shared memory (4 / 8 / 16 elements).
template <typename T>
__device__ __forceinline__ void unpack16(const uint4& u, float* dst)
{
    if constexpr (sizeof(T) == 1) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            // byte b of w -> float 2^23 + b, minus 2^23 (exact)
            const float2 lo = make_float2(__int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7650)),
                                          __int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7651)));
            const float2 hi = make_float2(__int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7652)),
                                          __int_as_float(__byte_perm(w[k], 0x4B000000u, 0x7653)));
            const float2 M = make_float2(-8388608.0f, -8388608.0f);
            const float2 a = __fadd2_rn(lo, M), b = __fadd2_rn(hi, M);
            *reinterpret_cast<float4*>(dst + 4 * k) = make_float4(a.x, a.y, b.x, b.y);
        }
    } else if constexpr (sizeof(T) == 2) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
        float f[8];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            if constexpr (std::is_same<T, __half>::value) {
                const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
                f[2 * k] = v.x;
                f[2 * k + 1] = v.y;
            } else {
                const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
                f[2 * k] = v.x;
                f[2 * k + 1] = v.y;
            }
        }
        *reinterpret_cast<float4*>(dst) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(dst + 4) = make_float4(f[4], f[5], f[6], f[7]);
    } else {
        *reinterpret_cast<float4*>(dst) = make_float4(__uint_as_float(u.x), __uint_as_float(u.y),
                                                      __uint_as_float(u.z), __uint_as_float(u.w));
    }
}

template <int KT, int C, typename T>
__global__ void __launch_bounds__(kThreads)
k_stream(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const StreamCfg cfg,
         unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int TWE = cfg.tile_w;
    const int nq = TWE >> 2, rpp = kThreads / nq;
    const int tid = threadIdx.x, qx = tid % nq, ty = tid / nq;
    const int plane = blockIdx.z;
    const T* s = src + g.sp.offset(plane);
    T* d = dst + g.dp.offset(plane);

    const int64_t WoC = (int64_t)g.Wo * C;
    const int64_t e0 = (int64_t)blockIdx.x * TWE;
    const int nE = (int)min((int64_t)TWE, WoC - e0);
    const int yb = blockIdx.y * cfg.band_h;
    const int ye = min(g.Ho, yb + cfg.band_h);

    // Staged columns: source pixels [px_lo, px_hi] of the strip's taps,
    // unclamped. Position p of a staged row holds element base + p of the
    // source row, where columns outside the image hold the edge pixel's
    // channels (clamp-to-edge). In-image elements arrive in load units of
    // EPU elements starting at a0 (aligned); the columns left of the image
    // (px < 0) and right of it (px >= W) are filled separately.
    const int j_first = (int)(e0 / C), j_last = (int)((e0 + nE - 1) / C);
    const int px_lo = first_tap<KT>(j_first, g.W, g.Wo, g.coord);
    const int px_hi = first_tap<KT>(j_last, g.W, g.Wo, g.coord) + KT - 1;
    const int EPU = cfg.vec ? 16 / (int)sizeof(T) : 1;      // elements per load unit
    const int in_lo = max(px_lo, 0) * C, in_hi = (min(px_hi, g.W - 1) + 1) * C;
    const int a0 = (in_lo / EPU) * EPU;
    const int units = (in_hi - a0 + EPU - 1) / EPU;
    // base <= px_lo * C, and a0 - base a multiple of 4 so the vector stores
    // of the load units land on 16-byte boundaries of the staged row.
    const int base = a0 - ((max(0, a0 - px_lo * C) + 3) & ~3);
    const int lpad = max(0, -px_lo) * C;                 // elements left of the image
    const int rpad = max(0, px_hi - (g.W - 1)) * C;      // elements right of the image
    const int span = max(a0 + units * EPU, (px_hi + 1) * C) - base;
    const int u0 = a0 - base;                            // staged position of the first unit
    if (span > cfg.swe_max || (u0 & 3) || (cfg.swe_max & 3)) {   // uniform over the block
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }

    // Ring rows are padded by 4 floats per 16 elements, so the 16-byte
    // accesses of both passes spread over the shared-memory banks.
    const int HRS = TWE + TWE / 4;                         // ring row stride
    float* SR = sm;                                        // [rs_rows][swe_max]
    float* HR = SR + cfg.rs_rows * cfg.swe_max;            // [rh][HRS]
    float* RW = HR + cfg.rh * HRS;                         // [band_cap][KT]
    int* RB = reinterpret_cast<int*>(RW + cfg.band_cap * KT);      // [band_cap]
    const int hmask = cfg.rh - 1;
    if (ye - yb > cfg.band_cap) {   // uniform; the host sizes the table for the band
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }

    // Column taps of this thread's four elements of the horizontal pass,
    // qx + nq k (k = 0..3: consecutive lanes gather neighbouring staged
    // elements, so the loads avoid bank conflicts): staged position of the
    // first tap (tap q is q * C further) and the weights, paired for FP32x2.
    int off[4];
    float2 w01[KT], w23[KT];
    {
        float wx[4][KT];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int el = qx + nq * k;
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

    // Staging of nn source rows starting at absolute row r0 into SR rows
    // 0..nn-1 (row indices clamped to the image).
    const int64_t pitch = g.src_pitch;
    // u -> (row k, unit w) of a staging work list: multiply-high by
    // ceil(2^32 / units) is exact for u * units < 2^32.
    const uint32_t umul = units > 1 ? 0xFFFFFFFFu / (uint32_t)units + 1u : 0u;
    auto split = [&](int u, int& k, int& w) {
        k = units > 1 ? (int)__umulhi((uint32_t)u, umul) : u;
        w = u - k * units;
    };
    auto row_ptr = [&](int r0, int k) -> const T* {
        return s + (int64_t)clampi(r0 + k, g.H) * pitch;
    };
    auto stage_pads = [&](int r0, int nn) {   // edge columns outside the image
        const int npad = lpad + rpad;
        for (int u = tid; u < nn * npad; u += kThreads) {
            const int k = u / npad, p = u - k * npad;
            const int c = p % C;
            const int src_el = p < lpad ? c : (g.W - 1) * C + c;
            const int pos = p < lpad ? (px_lo * C - base) + p : (g.W * C - base) + (p - lpad);
            SR[k * cfg.swe_max + pos] = Store<T>::load(row_ptr(r0, k) + src_el);
        }
    };
    uint4 pf[kPrefetch];
    auto issue = [&](int r0, int nn) {       // loads into registers (vector path)
        #pragma unroll
        for (int i = 0; i < kPrefetch; ++i) {
            const int u = tid + i * kThreads;
            if (u < nn * units) {
                int k, w;
                split(u, k, w);
                pf[i] = __ldg(reinterpret_cast<const uint4*>(row_ptr(r0, k) + a0 + w * EPU));
            }
        }
    };
    auto commit = [&](int r0, int nn) {     // registers -> FP32 rows
        #pragma unroll
        for (int i = 0; i < kPrefetch; ++i) {
            const int u = tid + i * kThreads;
            if (u < nn * units) {
                int k, w;
                split(u, k, w);
                unpack16<T>(pf[i], SR + k * cfg.swe_max + u0 + w * EPU);
            }
        }
        if (lpad + rpad) stage_pads(r0, nn);
    };
    auto stage_sync = [&](int r0, int nn) { // any alignment, any size
        const int total = nn * units;
        if (cfg.vec) {
            for (int b0 = 0; b0 < total; b0 += kPrefetch * kThreads) {
                #pragma unroll
                for (int i = 0; i < kPrefetch; ++i) {
                    const int u = b0 + tid + i * kThreads;
                    if (u < total) {
                        int k, w;
                split(u, k, w);
                        pf[i] = __ldg(reinterpret_cast<const uint4*>(row_ptr(r0, k) + a0 + w * EPU));
                    }
                }
                #pragma unroll
                for (int i = 0; i < kPrefetch; ++i) {
                    const int u = b0 + tid + i * kThreads;
                    if (u < total) {
                        int k, w;
                split(u, k, w);
                        unpack16<T>(pf[i], SR + k * cfg.swe_max + u0 + w * EPU);
                    }
                }
            }
        } else {
            for (int b0 = 0; b0 < total; b0 += 4 * kThreads) {
                float v[4];
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = b0 + tid + i * kThreads;
                    if (u < total) {
                        int k, w;
                split(u, k, w);
                        v[i] = Store<T>::load(row_ptr(r0, k) + a0 + w);
                    }
                }
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = b0 + tid + i * kThreads;
                    if (u < total) {
                        int k, w;
                split(u, k, w);
                        SR[k * cfg.swe_max + u0 + w] = v[i];
                    }
                }
            }
        }
        if (lpad + rpad) stage_pads(r0, nn);
    };
    // Row taps of the whole band, once: biased first tap row (with a flag
    // for rows whose weights select a single row exactly) and KT weights.
    for (int i = tid; i < ye - yb; i += kThreads) {
        float w[KT];
        const int f = taps<KT>(yb + i, g.H, g.Ho, g.coord, g.a, w);
        bool copy = false;
        if (KT == 4) copy = (w[0] == 0.0f && w[1] == 1.0f && w[2] == 0.0f && w[3] == 0.0f);
        if (KT == 2) copy = (w[0] == 1.0f && w[1] == 0.0f);
        if (KT == 1) copy = true;
        RB[i] = ((f + kRowBias) << 1) | (copy ? 1 : 0);
        #pragma unroll
        for (int p = 0; p < KT; ++p) RW[i * KT + p] = w[p];
    }
    __syncthreads();
    auto chunk_rows = [&](int y, int& lo, int& hi) {
        const int nR = min(cfg.chunk_h, ye - y);
        lo = (RB[y - yb] >> 1) - kRowBias;
        hi = (RB[y + nR - 1 - yb] >> 1) - kRowBias + KT - 1;
    };
    const int pf_cap = kPrefetch * kThreads;

    int lo, hi;
    chunk_rows(yb, lo, hi);
    int n_lo = lo, n_hi = hi;
    bool prefetched = false;
    if (cfg.vec && (n_hi - n_lo + 1) * units <= pf_cap) {
        issue(n_lo, n_hi - n_lo + 1);
        prefetched = true;
    }
    for (int y = yb; y < ye; y += cfg.chunk_h) {
        const int nR = min(cfg.chunk_h, ye - y);
        const int nn = n_hi - n_lo + 1;
        if (nn > cfg.rs_rows) {   // uniform; cannot happen with host bounds
            if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
            return;
        }
        const float* rw = RW + (y - yb) * KT;
        const int* rb = RB + (y - yb);
        // Source rows of this chunk.
        if (prefetched) commit(n_lo, nn); else stage_sync(n_lo, nn);
        __syncthreads();

        // Prefetch the next chunk's new rows.
        int nx_lo = 0, nx_hi = -1;
        bool nx_pref = false;
        if (y + cfg.chunk_h < ye) {
            chunk_rows(y + cfg.chunk_h, lo, hi);
            nx_lo = max(n_hi + 1, lo);
            nx_hi = hi;
            if (cfg.vec && (nx_hi - nx_lo + 1) * units <= pf_cap) {
                issue(nx_lo, nx_hi - nx_lo + 1);
                nx_pref = true;
            }
        }

        // Horizontal pass over the new rows.
        if (qx < nE) {
            for (int k = ty; k < nn; k += rpp) {
                const float* Sr = SR + k * cfg.swe_max;
                float2 h01 = make_float2(0.0f, 0.0f), h23 = make_float2(0.0f, 0.0f);
                #pragma unroll
                for (int q = 0; q < KT; ++q) {
                    h01 = __ffma2_rn(w01[q], make_float2(Sr[off[0] + q * C], Sr[off[1] + q * C]), h01);
                    h23 = __ffma2_rn(w23[q], make_float2(Sr[off[2] + q * C], Sr[off[3] + q * C]), h23);
                }
                float* hr = HR + ((n_lo + k + kRowBias) & hmask) * HRS;
                hr[hpos(qx)] = h01.x;
                hr[hpos(qx + nq)] = h01.y;
                hr[hpos(qx + 2 * nq)] = h23.x;
                hr[hpos(qx + 3 * nq)] = h23.y;
            }
        }
        __syncthreads();

        // Vertical pass and store: each thread writes 16 bytes (EV
        // consecutive elements) of one output row per iteration.
        {
            constexpr int EV = 16 / (int)sizeof(T);
            constexpr int NG = EV / 4;
            const int nv = TWE / EV, vpp = kThreads / nv;
            const int vx = tid % nv, vy = tid / nv;
            const int ev0 = EV * vx;
            if (ev0 < nE) {
                const int cnt = min(EV, nE - ev0);
                const int hoff = hpos(ev0);
                for (int i = vy; i < nR; i += vpp) {
                    const int code = rb[i];
                    const int f = code >> 1;             // biased first tap row
                    float2 v[2 * NG];
                    if (code & 1) {
                        const float* hr = HR + ((f + (KT == 4 ? 1 : 0)) & hmask) * HRS + hoff;
                        #pragma unroll
                        for (int gq = 0; gq < NG; ++gq) {
                            const float4 hv = *reinterpret_cast<const float4*>(hr + 4 * gq);
                            v[2 * gq] = make_float2(hv.x, hv.y);
                            v[2 * gq + 1] = make_float2(hv.z, hv.w);
                        }
                    } else {
                        float wy[KT];
                        if constexpr (KT == 4) {
                            const float4 w4 = *reinterpret_cast<const float4*>(rw + i * 4);
                            wy[0] = w4.x; wy[1] = w4.y; wy[2] = w4.z; wy[3] = w4.w;
                        } else {
                            #pragma unroll
                            for (int p = 0; p < KT; ++p) wy[p] = rw[i * KT + p];
                        }
                        #pragma unroll
                        for (int gq = 0; gq < 2 * NG; ++gq) v[gq] = make_float2(0.0f, 0.0f);
                        #pragma unroll
                        for (int p = 0; p < KT; ++p) {
                            const float2 w2 = make_float2(wy[p], wy[p]);
                            const float* hr = HR + ((f + p) & hmask) * HRS + hoff;
                            #pragma unroll
                            for (int gq = 0; gq < NG; ++gq) {
                                const float4 hv = *reinterpret_cast<const float4*>(hr + 4 * gq);
                                v[2 * gq] = __ffma2_rn(w2, make_float2(hv.x, hv.y), v[2 * gq]);
                                v[2 * gq + 1] = __ffma2_rn(w2, make_float2(hv.z, hv.w), v[2 * gq + 1]);
                            }
                        }
                    }
                    store16<T>(d + (int64_t)(y + i) * g.dst_pitch + e0 + ev0, v, cnt);
                }
            }
        }
        n_lo = nx_lo;
        n_hi = nx_hi;
        prefetched = nx_pref;
    }
}

// ---------------------------------------------------------------------------
// Host side

static int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

bool stream_config(const Geom& g, int method, int dtype, const void* src, StreamCfg& c)
{
    const int KT = method_taps(method);
    const int es = (int)dtype_size(dtype);
    // strips of a multiple of 16 elements: 4 per thread in the horizontal
    // pass, 16 bytes per thread in the vertical pass
    if (c.tile_w < 16 || (c.tile_w & 15) || c.tile_w / 4 > kThreads || kThreads % (c.tile_w / 4)) return false;
    if (c.tile_w / (16 / es) > kThreads || kThreads % (c.tile_w / (16 / es))) return false;
    if (c.chunk_h < 1) return false;
    // 16-byte units need every staged row to start and end on 16 bytes.
    const uintptr_t base = reinterpret_cast<uintptr_t>(src);
    const bool planar = g.sp.cp > 1 || g.planes > 1;
    c.vec = (base % 16 == 0) && ((g.src_pitch * es) % 16 == 0) && (((int64_t)g.W * g.C * es) % 16 == 0) &&
            (!planar || ((g.sp.n_stride * es) % 16 == 0 && (g.sp.c_stride * es) % 16 == 0)) ? 1 : 0;
    const int EPU = c.vec ? 16 / es : 1;
    const int kpx = (c.tile_w + g.C - 1) / g.C + 1;
    const int span_px = tap_span_bound(kpx, g.W, g.Wo, KT, g.coord);
    // Unclamped footprint, the alignment margin of the first load unit (<
    // EPU) and the rounding of the row base to 4 elements (< 4).
    c.swe_max = ((span_px * g.C + 2 * EPU + 4) + 3) & ~3;
    const int span_rows = tap_span_bound(c.chunk_h, g.H, g.Ho, KT, g.coord);
    c.rh = next_pow2(span_rows);
    c.rs_rows = span_rows;
    // Band row table: at most kMaxBand rows (a multiple of chunk_h).
    const int chunks_cap = std::max(1, kMaxBand / c.chunk_h);
    c.band_cap = (int)std::min<int64_t>((int64_t)chunks_cap * c.chunk_h,
                                        ((int64_t)g.Ho + c.chunk_h - 1) / c.chunk_h * c.chunk_h);
    c.smem = sizeof(float) * ((size_t)c.rs_rows * c.swe_max + (size_t)c.rh * (c.tile_w + c.tile_w / 4) +
                              (size_t)c.band_cap * KT) +
             sizeof(int) * (size_t)c.band_cap;
    return c.smem <= max_smem_per_block();
}

template <int KT, int C, typename T>
static void* stream_func() { return reinterpret_cast<void*>(&k_stream<KT, C, T>); }

template <int KT, typename T>
static void* stream_func_c(int C)
{
    switch (C) {
    case 1: return stream_func<KT, 1, T>();
    case 2: return stream_func<KT, 2, T>();
    case 3: return stream_func<KT, 3, T>();
    default: return stream_func<KT, 4, T>();
    }
}

template <typename T>
static void* stream_func_m(int method, int C)
{
    switch (method) {
    case M_NEAREST: return stream_func_c<1, T>(C);
    case M_BILINEAR: return stream_func_c<2, T>(C);
    default: return stream_func_c<4, T>(C);
    }
}

static void* stream_kernel(int method, int dtype, int C)
{
    switch (dtype) {
    case DT_U8: return stream_func_m<uint8_t>(method, C);
    case DT_F16: return stream_func_m<__half>(method, C);
    case DT_BF16: return stream_func_m<__nv_bfloat16>(method, C);
    default: return stream_func_m<float>(method, C);
    }
}

// Band height: enough bands for about `waves` blocks per resident slot.
static int choose_band(const Geom& g, const StreamCfg& c, int per_sm, int waves)
{
    const int64_t strips = ((int64_t)g.Wo * g.C + c.tile_w - 1) / c.tile_w;
    const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
    const int64_t want = std::max<int64_t>(1, resident * waves / (strips * g.planes));   // no partial extra wave
    const int64_t chunks = (g.Ho + c.chunk_h - 1) / c.chunk_h;
    const int64_t bands = std::min<int64_t>(want, chunks);
    const int64_t chunks_per_band = std::min<int64_t>((chunks + bands - 1) / bands, c.band_cap / c.chunk_h);
    return (int)(std::max<int64_t>(1, chunks_per_band) * c.chunk_h);
}

cudaError_t launch_stream(const Geom& g, int method, int dtype, const void* src, void* dst, StreamCfg c,
                          cudaStream_t st)
{
    void* func = stream_kernel(method, dtype, g.C);
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, kThreads, c.band_h <= 0 ? &per_sm : nullptr);
    if (e != cudaSuccess) return e;
    if (c.band_h <= 0) {
        c.band_h = choose_band(g, c, per_sm, c.waves > 0 ? c.waves : 4);
    }
    dim3 grid((unsigned)(((int64_t)g.Wo * g.C + c.tile_w - 1) / c.tile_w),
              (unsigned)((g.Ho + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &c, &fw};
    e = cudaLaunchKernel(func, grid, dim3(kThreads), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

StreamCfg stream_default(const Geom& g, int method, int dtype, const void* src)
{
    // 512-element strips, the tallest chunk (<= 16 rows) within 64 KB of
    // shared memory, else the largest that fits at all.
    for (int pass = 0; pass < 2; ++pass) {
        for (int tw : {512, 256, 128}) {
            for (int ch = 16; ch >= 1; ch >>= 1) {
                StreamCfg c{};
                c.tile_w = tw;
                c.chunk_h = ch;
                if (!stream_config(g, method, dtype, src, c)) continue;
                if (pass == 0 && c.smem > 64 * 1024) continue;
                return c;
            }
        }
    }
    return StreamCfg{};
}

}  // namespace rs
