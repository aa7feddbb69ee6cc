// Register-window resampling (bilinear / bicubic): the per-block work.
//
// A block owns a strip of tile_w = 4 * 256 output elements and a band of
// output rows; thread t owns strip elements t, t + 256, t + 512 and t + 768
// for the whole band and walks down it (consecutive lanes then gather
// neighbouring source elements: no shared-memory bank conflicts). Output row i of the band takes source rows
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
// renaming. Source rows are staged in chunks of R rows as FP32 (double
// buffered). With 16-byte-aligned rows the raw bytes of chunks c + 1 and
// c + 2 are already on their way (cp.async into a three-slot raw ring) while
// chunk c is processed; each thread converts the units it copied itself, so
// one barrier per chunk suffices. Out-of-image rows and columns take the
// edge pixel.
#pragma once

#include <algorithm>
#include <type_traits>

#include "rs_common.cuh"

namespace rs {

static constexpr int kPolyThreads = 256;
static constexpr int kPolyElems = 4 * kPolyThreads;   // strip width in elements
static constexpr int kPolyMaxBand = 256;              // rows of the row-tap table

// Stores a thread's four outputs (a.x, a.y, b.x, b.y) at p, p + 256,
// p + 512 and p + 768; only the first `nact` exist (ragged strip end).
template <typename T>
__device__ __forceinline__ void poly_store_strided(T* p, float2 a, float2 b, int nact)
{
    constexpr int S = kPolyThreads;
    if constexpr (sizeof(T) == 1) {
        // Round to nearest even and saturate to [0, 255] in one conversion.
        const float v[4] = {a.x, a.y, b.x, b.y};
        uint8_t* q = reinterpret_cast<uint8_t*>(p);
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < nact) {
                unsigned short r;
                asm("cvt.rni.sat.u8.f32 %0, %1;" : "=h"(r) : "f"(v[k]));
                q[k * S] = (uint8_t)r;
            }
        }
    } else if constexpr (sizeof(T) == 2) {
        uint32_t lo, hi;
        if constexpr (std::is_same<T, __half>::value) {
            __half2 h0 = __float22half2_rn(a), h1 = __float22half2_rn(b);
            lo = *reinterpret_cast<uint32_t*>(&h0);
            hi = *reinterpret_cast<uint32_t*>(&h1);
        } else {
            __nv_bfloat162 h0 = __float22bfloat162_rn(a), h1 = __float22bfloat162_rn(b);
            lo = *reinterpret_cast<uint32_t*>(&h0);
            hi = *reinterpret_cast<uint32_t*>(&h1);
        }
        uint16_t* q = reinterpret_cast<uint16_t*>(p);
        const uint16_t v[4] = {(uint16_t)lo, (uint16_t)(lo >> 16), (uint16_t)hi, (uint16_t)(hi >> 16)};
        #pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < nact) q[k * S] = v[k];
    } else {
        const float v[4] = {a.x, a.y, b.x, b.y};
        #pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < nact) p[k * S] = v[k];
    }
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

__device__ __forceinline__ float raw_to_float(uint8_t v) { return (float)v; }
__device__ __forceinline__ float raw_to_float(__half v) { return __half2float(v); }
__device__ __forceinline__ float raw_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float raw_to_float(float v) { return v; }

// The work of one block: strip bx (1024 output elements) and band by of
// one plane (s, d already point at the plane). Used by the single-image
// kernel and by the persistent batched kernel. FIX = 2: every position of
// the band emits exactly two output rows (the asymmetric map at exactly x2,
// bands of an even number of rows from an even row), so the emit step needs
// neither the per-position row count nor a loop; the block checks this
// against its row taps and reports a fault instead of computing otherwise.
template <int KT, int C, typename T, int MODE, int FIX = 0>
__device__ __forceinline__ void poly_body(const Geom& g, const T* __restrict__ s, T* __restrict__ d,
                                          const PolyCfg& cfg, int bx, int by, float* sm, unsigned int* fault)
{
    static_assert(MODE == 1 || MODE == 2, "staging mode: 1 aligned units, 2 shifted blocks");
    static_assert(FIX == 0 || FIX == 2, "rows per position: 0 any (table), 2 exactly two");
    const int tid = threadIdx.x;

    const int64_t WoC = (int64_t)g.Wo * C;
    const int64_t e0 = (int64_t)bx * kPolyElems;
    const int nE = (int)min((int64_t)kPolyElems, WoC - e0);
    const int yb = by * cfg.band_h;
    const int ye = min(g.Ho, yb + cfg.band_h);
    const int nrows = ye - yb;

    // Staged columns (as in the streaming kernel): source pixels
    // [px_lo, px_hi] unclamped; position p of a staged row holds element
    // base + p; in-image elements arrive in units of EPU elements from a0,
    // out-of-image columns hold the edge pixel.
    const int j_first = (int)(e0 / C), j_last = (int)((e0 + nE - 1) / C);
    const int px_lo = first_tap<KT>(j_first, g.W, g.Wo, g.coord);
    const int px_hi = first_tap<KT>(j_last, g.W, g.Wo, g.coord) + KT - 1;
    constexpr int EPU = 16 / (int)sizeof(T);
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
    int* NC = RF + cfg.band_cap;                           // [pos_cap] rows per position
    // Raw 16-byte load units of the next two chunks (vector path): [3][R][raw_row].
    unsigned char* RAW = reinterpret_cast<unsigned char*>(sm) + cfg.raw_off;
    // MODE 1: 16-byte-aligned rows, each unit copied and converted by one
    // thread; MODE 2 (shifted): rows at any element alignment, copied as the
    // aligned 16-byte blocks around them (units + 1 per row) and realigned
    // when converted.
    constexpr bool shifted = MODE == 2;
    if (cfg.vec != MODE || (units + (shifted ? 2 : 0)) * 16 > cfg.raw_row) {   // uniform; the host sizes raw rows
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }

    // Row taps of the band.
    for (int i = tid; i < nrows; i += kPolyThreads) {
        float w[KT];
        RF[i] = taps<KT>(yb + i, g.H, g.Ho, g.coord, g.a, w);
        #pragma unroll
        for (int p = 0; p < KT; ++p) RW[i * KT + p] = w[p];
    }

    // Column taps of this thread's four elements tid + 256 k (the first
    // nact of them lie inside the strip).
    const int nact = max(0, min(4, (nE - tid + kPolyThreads - 1) / kPolyThreads));
    int off[4];
    float2 w01[KT], w23[KT];
    {
        float wx[4][KT];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int el = tid + kPolyThreads * k;
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
    // Vector path: cp.async copies of 16-byte units into raw slot `slot`,
    // one commit group per chunk. Each thread later converts exactly the
    // units it copied, so its own wait_group makes them visible to it.
    auto issue_async = [&](int r0, int nn, int slot) {
        unsigned char* rb = RAW + (size_t)slot * R * cfg.raw_row;
        for (int u = tid; u < nn * units; u += kPolyThreads) {
            int k, w;
            split(u, k, w);
            const T* gsrc = row_ptr(r0 + k) + a0 + w * EPU;
            const unsigned sdst = (unsigned)__cvta_generic_to_shared(rb + k * cfg.raw_row + w * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(gsrc) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto convert = [&](int r0, int nn, int slot, float* dstb) {
        const unsigned char* rb = RAW + (size_t)slot * R * cfg.raw_row;
        for (int u = tid; u < nn * units; u += kPolyThreads) {
            int k, w;
            split(u, k, w);
            const uint4 v = *reinterpret_cast<const uint4*>(rb + k * cfg.raw_row + w * 16);
            poly_unpack16<T>(v, dstb + k * cfg.swe_max + u0 + w * EPU);
        }
        if (lpad + rpad) pads(r0, nn, dstb);
    };
    // Shifted path. Row k of a chunk starts its raw copy at the aligned
    // block A below its first staged byte Rb = &row[a0] (phase Rb - A < 16)
    // and copies units + 1 blocks. A block not wholly inside the plane (the
    // first row's head, the last row's tail) is filled element by element
    // instead, only with the staged elements it holds.
    const uintptr_t plane_lo = reinterpret_cast<uintptr_t>(s);
    const uintptr_t plane_hi = reinterpret_cast<uintptr_t>(s + (int64_t)(g.H - 1) * g.src_pitch + (int64_t)g.W * C);
    const uint32_t umul1 = 0xFFFFFFFFu / (uint32_t)(units + 1) + 1u;
    auto issue_shifted = [&](int r0, int nn, int slot) {
        unsigned char* rb = RAW + (size_t)slot * R * cfg.raw_row;
        const int per = units + 1;
        for (int u = tid; u < nn * per; u += kPolyThreads) {
            const int k = (int)__umulhi((uint32_t)u, umul1), w = u - k * per;
            const uintptr_t rb0 = reinterpret_cast<uintptr_t>(row_ptr(r0 + k) + a0);
            const uintptr_t blk = (rb0 & ~(uintptr_t)15) + 16 * (uintptr_t)w;
            unsigned char* dsts = rb + k * cfg.raw_row + w * 16;
            if (blk >= plane_lo && blk + 16 <= plane_hi) {
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(dsts);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst),
                             "l"(reinterpret_cast<const void*>(blk)) : "memory");
            } else {
                const int phase = (int)(rb0 & 15);
                // staged elements a0 + e with byte offset phase + e * es in [16 w, 16 w + 16)
                const int es = (int)sizeof(T);
                const int e_lo = max(0, (16 * w - phase + es - 1) / es);
                const int e_hi = min(in_hi - a0, (16 * w + 16 - phase) / es);
                const T* rowp = row_ptr(r0 + k) + a0;
                for (int e = e_lo; e < e_hi; ++e)
                    *reinterpret_cast<T*>(rb + k * cfg.raw_row + phase + e * es) = rowp[e];
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // Converts the staged groups of EPU elements of every row (any thread
    // any group: a barrier precedes it), realigning by the row's phase.
    auto convert_shifted = [&](int r0, int nn, int slot, float* dstb) {
        const unsigned char* rb = RAW + (size_t)slot * R * cfg.raw_row;
        const int valid = in_hi - a0;   // staged elements per row
        for (int u = tid; u < nn * units; u += kPolyThreads) {
            int k, w;
            split(u, k, w);
            const int phase = (int)(reinterpret_cast<uintptr_t>(row_ptr(r0 + k) + a0) & 15);
            const uint32_t* W = reinterpret_cast<const uint32_t*>(rb + k * cfg.raw_row) + (phase >> 2) + 4 * w;
            const int sh = 8 * (phase & 3);
            uint32_t x[5];
            #pragma unroll
            for (int q = 0; q < 5; ++q) x[q] = W[q];
            uint4 v;
            v.x = __funnelshift_r(x[0], x[1], sh);
            v.y = __funnelshift_r(x[1], x[2], sh);
            v.z = __funnelshift_r(x[2], x[3], sh);
            v.w = __funnelshift_r(x[3], x[4], sh);
            float* dp = dstb + k * cfg.swe_max + u0 + w * EPU;
            if (w * EPU + EPU <= valid) {
                poly_unpack16<T>(v, dp);
            } else {   // the row's last group: positions past the image hold pads
                const T* e = reinterpret_cast<const T*>(rb + k * cfg.raw_row + phase) + w * EPU;
                for (int q = 0; w * EPU + q < valid; ++q) dp[q] = raw_to_float(e[q]);
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

    for (int p = tid; p < cfg.pos_cap; p += kPolyThreads) NC[p] = 0;
    __syncthreads();   // row taps visible
    const int b_first = RF[0];
    const int b_last = RF[nrows - 1];
    if (b_last - b_first + 1 > cfg.pos_cap) {   // uniform; the host bounds the positions
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    // Number of output rows at each position (runs of equal first taps).
    for (int i0 = tid; i0 < nrows; i0 += kPolyThreads) {
        if (i0 == 0 || RF[i0] != RF[i0 - 1]) {
            int len = 1;
            while (i0 + len < nrows && RF[i0 + len] == RF[i0]) ++len;
            NC[RF[i0] - b_first] = len;
        }
    }
    if constexpr (FIX == 2) {   // uniform; before any copy is issued
        bool ok = (nrows % 2) == 0;
        for (int q = tid; 2 * q < nrows; q += kPolyThreads)
            ok = ok && RF[2 * q + 1] == RF[2 * q] && (2 * q + 2 >= nrows || RF[2 * q + 2] == RF[2 * q] + 1);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
            return;
        }
    }
    // Source rows in order: b_first .. b_last + KT - 1, in chunks of R.
    const int r_first = b_first, r_end = b_last + KT;      // [r_first, r_end)
    auto chunk_rows = [&](int c) { return max(0, min(R, r_end - (r_first + c * R))); };
    int cidx = 0;                                          // current chunk
    int chunk_lo = r_first;
    int nn = chunk_rows(0);
    if constexpr (shifted) {
        issue_shifted(r_first, nn, 0);
        issue_shifted(r_first + R, chunk_rows(1), 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        convert_shifted(r_first, nn, 0, SR);
    } else {
        issue_async(r_first, nn, 0);
        issue_async(r_first + R, chunk_rows(1), 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        convert(r_first, nn, 0, SR);
    }
    __syncthreads();
    if constexpr (shifted) issue_shifted(r_first + 2 * R, chunk_rows(2), 2);
    else issue_async(r_first + 2 * R, chunk_rows(2), 2);
    int half = 0;

    // Register window: h[p] holds source row (b + p) at position b.
    float2 h01[KT], h23[KT];
    int i = 0;                 // next output row of the band
    int b = b_first;           // current position
    // Prime rows b_first .. b_first + KT - 2 (all in the first chunk: R >= KT).
    #pragma unroll
    for (int p = 0; p < KT - 1; ++p) hrow(SR + p * cfg.swe_max, h01[p], h23[p]);
    int r = b_first + KT - 1;  // next source row to interpolate (newest window row)

    // Blend output row `row` from window slots slot[0..KT) with its weights.
    auto blend = [&](int row, const int* slot, float2& v01, float2& v23) {
        float wy[KT];
        if constexpr (KT == 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(RW + 4 * row);
            wy[0] = w4.x; wy[1] = w4.y; wy[2] = w4.z; wy[3] = w4.w;
        } else {
            const float2 w2 = *reinterpret_cast<const float2*>(RW + 2 * row);
            wy[0] = w2.x; wy[1] = w2.y;
        }
        v01 = make_float2(0.0f, 0.0f);
        v23 = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int p = 0; p < KT; ++p) {
            const float2 w2 = make_float2(wy[p], wy[p]);
            v01 = __ffma2_rn(w2, h01[slot[p]], v01);
            v23 = __ffma2_rn(w2, h23[slot[p]], v23);
        }
    };
    // Output rows are addressed from the band's first row with 32-bit
    // offsets (the host bounds band_cap * dst_pitch below 2^31).
    T* const dband = d + (int64_t)yb * g.dst_pitch + e0 + tid;
    const int pitch32 = (int)g.dst_pitch;
    auto put = [&](int row, float2 v01, float2 v23) {
        if (nact > 0) poly_store_strided<T>(dband + row * pitch32, v01, v23, nact);
    };
    // Emit the output rows whose first tap is b (two at a time: independent
    // chains), from window slots slot[0..KT).
    auto emit = [&](const int* slot) {
        if constexpr (FIX == 2 && std::is_same<T, uint8_t>::value) {
            // The band starts on an even row, so row i has t = 0 and the
            // weights (0, 1, 0, 0) (bilinear (1, 0)); with finite values (all
            // uint8 data) the blend returns the window row itself, up to the
            // sign of a zero, which the byte conversion does not see.
            constexpr int s1 = KT == 4 ? 1 : 0;
            float2 c01, c23;
            blend(i + 1, slot, c01, c23);
            put(i, h01[slot[s1]], h23[slot[s1]]);
            put(i + 1, c01, c23);
            i += 2;
        } else if constexpr (FIX == 2) {
            float2 a01, a23, c01, c23;
            blend(i, slot, a01, a23);
            blend(i + 1, slot, c01, c23);
            put(i, a01, a23);
            put(i + 1, c01, c23);
            i += 2;
        } else {
            const int nb = NC[b - b_first];
            int k = 0;
            for (; k + 1 < nb; k += 2) {
                float2 a01, a23, c01, c23;
                blend(i + k, slot, a01, a23);
                blend(i + k + 1, slot, c01, c23);
                put(i + k, a01, a23);
                put(i + k + 1, c01, c23);
            }
            if (k < nb) {
                float2 a01, a23;
                blend(i + k, slot, a01, a23);
                put(i + k, a01, a23);
            }
            i += nb;
        }
    };

    while (b <= b_last) {
        #pragma unroll
        for (int u = 0; u < KT; ++u) {
            if (b <= b_last) {
                // Make source row r = b + KT - 1 available in the staged chunk.
                // Chunk c starts at row r_first + c R and r = b + KT - 1 starts
                // at r_first + KT - 1, so with R a multiple of KT (the host's
                // rule) a chunk is entered only at u == 1: one copy of the
                // switch code per unrolled group.
                if (u == 1 && r >= chunk_lo + nn) {
                    // Move to chunk c = cidx + 1. Its FP32 half held chunk c-2,
                    // whose reads all precede the barrier of the previous
                    // switch; its raw slot was filled two switches ago (wait
                    // for this thread's copies, at most one newer group may
                    // still be in flight). The barrier publishes the chunk;
                    // then chunk c+2 is issued into the raw slot of chunk c-1,
                    // which this thread has already converted.
                    ++cidx;
                    half ^= 1;
                    chunk_lo = r_first + cidx * R;
                    nn = chunk_rows(cidx);
                    float* dstb = SR + half * R * cfg.swe_max;
                    if constexpr (shifted) {
                        // every thread's copies must land before any converts
                        asm volatile("cp.async.wait_group 1;" ::: "memory");
                        __syncthreads();
                        convert_shifted(chunk_lo, nn, cidx % 3, dstb);
                    } else {
                        asm volatile("cp.async.wait_group 1;" ::: "memory");
                        convert(chunk_lo, nn, cidx % 3, dstb);
                    }
                    __syncthreads();
                    if constexpr (shifted) issue_shifted(r_first + (cidx + 2) * R, chunk_rows(cidx + 2), (cidx + 2) % 3);
                    else issue_async(r_first + (cidx + 2) * R, chunk_rows(cidx + 2), (cidx + 2) % 3);
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

}  // namespace rs
