// Register-window resampling (bilinear / bicubic): the per-block work of the
// forward window kernel and of the batch's window items.
//
// A block of kWinThreads threads owns a strip of SP = kWinThreads * P output
// pixels (all C channels) and a band of output rows; each thread owns P
// pixels of the strip for the whole band.
//
// Output row i of the band takes source rows f(i) .. f(i) + KT - 1 (Eqs.
// 2-3; f never decreases with i). The thread keeps the horizontally
// interpolated values of the last KT source rows at its pixels in registers
// (the window) and walks a source-row position b down the band: at position
// b it interpolates source row b + KT - 1 into the window, then blends every
// output row with f(i) == b from registers. The position loop is unrolled KT
// times so the window rotates by register renaming. Every sum runs over the
// taps in order from the first, starting at zero, as in every kernel of the
// library.
//
// Two forms:
//  - general (any scale): warp w of the block owns the 32 P pixels
//    js = strip start + 32 P w .., and lane l the pixels js + l + 32 m
//    (m < P). Source rows are staged channel-planar in FP32, so consecutive
//    lanes gather neighbouring (or the same) staged samples: the tap loads
//    have no shared-memory bank conflicts. Pixels m, m + 1 pair up in packed
//    FP32x2 FMAs (one tap of one channel for two pixels per instruction);
//    every stored element is one store of its own.
//  - X2 (the asymmetric map at exactly x2 on both axes): output pixel 2u has
//    t = 0 (weights (0, 1, 0, 0), bilinear (1, 0)), so it is the source
//    sample itself; pixel 2u + 1 has t = 1/2 and the same weights for every
//    u. Thread t owns the P consecutive pixels strip start + t P .., which
//    read P/2 + KT - 1 consecutive source pixels: loaded once per source row
//    with vector loads from interleaved FP32 rows, only the odd pixels are
//    interpolated, every even output row is a window row and every odd one a
//    blend with the t = 1/2 weights (with finite inputs: the general form's
//    results up to the sign of a zero). A thread's row leaves as one to
//    three 4-, 8- or 16-byte stores.
//
// Staging: source rows are copied in chunks of R rows as the 16-byte-aligned
// global blocks around each row's footprint (cp.async). The general form
// keeps a two-slot raw ring (the next chunk in flight while the current one
// is used) and widens each landed chunk to channel-planar FP32 rows, one warp
// per row and one pixel per lane, realigning by the row's byte phase;
// positions outside the image read the edge pixel. Two barriers per chunk:
// one before the FP32 rows are overwritten, one after. The exact-x2 form
// reads its footprints from the raw rows directly (see win_body_x2).
#pragma once

#include <type_traits>

#include "rs_common.cuh"

namespace rs {

static constexpr int kWinThreads = 128;
static constexpr int kWinWarps = kWinThreads / 32;
static constexpr int kWinMaxBand = 256;   // rows of the per-block row-tap tables

template <int C, typename T, bool X2>
struct WinShape {
    static constexpr int es = (int)sizeof(T);
    // X2: a contiguous run of 8 to 32 bytes per output row, at most 12
    // elements; general: P pixels strided by 32 (at most 12 elements).
    static constexpr int P = X2 ? (C == 1 ? (es == 4 ? 4 : 8) : C == 2 ? (es == 4 ? 2 : 4) : C == 3 ? (es == 1 ? 4 : 2) : 2)
                                : (C == 1 ? 8 : C == 4 ? 2 : 4);
    static constexpr int NP = P / 2;                 // pixel pairs
    static constexpr int E = P * C;                  // elements per thread per row
    static constexpr int SP = kWinThreads * P;       // strip width in pixels
    // X2 run: bytes, 32-bit words and widest store unit per output row; the
    // staged floats between consecutive threads' footprints and the vector
    // width (floats) of their footprint loads.
    static constexpr int BYTES = E * es;
    static constexpr int NW = BYTES / 4;
    static constexpr int VU = BYTES % 16 == 0 ? 16 : BYTES % 8 == 0 ? 8 : 4;
    static constexpr int HALF = NP * C;
    static constexpr int VL = HALF % 4 == 0 ? 4 : HALF % 2 == 0 ? 2 : 1;
    static_assert(P % 2 == 0, "pixels pair up");
    static_assert(!X2 || BYTES % 4 == 0, "an X2 run is whole 32-bit words");
};

__device__ __forceinline__ float win_widen(uint8_t v) { return __uint_as_float(0x4B000000u | v) - 8388608.0f; }
__device__ __forceinline__ float win_widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float win_widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float win_widen(float v) { return v; }

// Four consecutive uint8 samples (one word, first sample in the low byte) to FP32.
__device__ __forceinline__ float4 win_widen4(uint32_t w)
{
    const float2 M = make_float2(-8388608.0f, -8388608.0f);
    const float2 lo = __fadd2_rn(make_float2(__int_as_float(__byte_perm(w, 0x4B000000u, 0x7650)),
                                             __int_as_float(__byte_perm(w, 0x4B000000u, 0x7651))), M);
    const float2 hi = __fadd2_rn(make_float2(__int_as_float(__byte_perm(w, 0x4B000000u, 0x7652)),
                                             __int_as_float(__byte_perm(w, 0x4B000000u, 0x7653))), M);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// uint8 store value: round to nearest even, saturate to [0, 255].
__device__ __forceinline__ uint32_t win_u8(float v)
{
    uint32_t b;
    asm("cvt.rni.sat.u8.f32 %0, %1;" : "=r"(b) : "f"(v));
    return b;
}

// X2: the E outputs of a thread's row, v[p][c] = (pixel 2p, pixel 2p + 1) of
// channel c, rounded to T and packed into words in memory order.
template <int C, typename T>
__device__ __forceinline__ void win_pack(const float2 (&v)[WinShape<C, T, true>::NP][C],
                                         uint32_t (&w)[WinShape<C, T, true>::NW])
{
    using S = WinShape<C, T, true>;
    constexpr int E = S::E;
    float x[E];
    #pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = e / C, c = e % C;
        x[e] = (k & 1) ? v[k >> 1][c].y : v[k >> 1][c].x;
    }
    if constexpr (sizeof(T) == 1) {
        #pragma unroll
        for (int q = 0; q < E / 4; ++q)
            w[q] = __byte_perm(__byte_perm(win_u8(x[4 * q]), win_u8(x[4 * q + 1]), 0x0040),
                               __byte_perm(win_u8(x[4 * q + 2]), win_u8(x[4 * q + 3]), 0x0040), 0x5410);
    } else if constexpr (sizeof(T) == 2) {
        #pragma unroll
        for (int q = 0; q < E / 2; ++q) {
            if constexpr (std::is_same<T, __half>::value) {
                const __half2 h = __floats2half2_rn(x[2 * q], x[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
        }
    } else {
        #pragma unroll
        for (int q = 0; q < E; ++q) w[q] = __float_as_uint(x[q]);
    }
}

// X2: stores a packed run at p with the widest stores its alignment allows.
template <int C, typename T>
__device__ __forceinline__ void win_store_run(T* p, const uint32_t (&w)[WinShape<C, T, true>::NW], int align)
{
    using S = WinShape<C, T, true>;
    constexpr int NW = S::NW;
    if (S::VU == 16 && align >= 16) {
        #pragma unroll
        for (int q = 0; q < NW / 4; ++q)
            reinterpret_cast<uint4*>(p)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else if (S::VU >= 8 && align >= 8) {
        #pragma unroll
        for (int q = 0; q < NW / 2; ++q) reinterpret_cast<uint2*>(p)[q] = make_uint2(w[2 * q], w[2 * q + 1]);
    } else if (align >= 4) {
        #pragma unroll
        for (int q = 0; q < NW; ++q) reinterpret_cast<uint32_t*>(p)[q] = w[q];
    } else if (align >= 2) {
        #pragma unroll
        for (int q = 0; q < NW; ++q) {
            reinterpret_cast<uint16_t*>(p)[2 * q] = (uint16_t)w[q];
            reinterpret_cast<uint16_t*>(p)[2 * q + 1] = (uint16_t)(w[q] >> 16);
        }
    } else {
        uint8_t* q = reinterpret_cast<uint8_t*>(p);
        #pragma unroll
        for (int e = 0; e < 4 * NW; ++e) q[e] = (uint8_t)(w[e >> 2] >> (8 * (e & 3)));
    }
}

// Fused pre-process (X2): P values of one channel plane, rounded to TO and
// packed into words in memory order.
template <int P, typename TO>
__device__ __forceinline__ void win_pack_plane(const float (&y)[P], uint32_t (&w)[P * sizeof(TO) / 4])
{
    if constexpr (sizeof(TO) == 4) {
        #pragma unroll
        for (int k = 0; k < P; ++k) w[k] = __float_as_uint(y[k]);
    } else {
        #pragma unroll
        for (int q = 0; q < P / 2; ++q) {
            if constexpr (std::is_same<TO, __half>::value) {
                const __half2 h = __floats2half2_rn(y[2 * q], y[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(y[2 * q], y[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
        }
    }
}

// NW words at p with the widest stores its alignment (align bytes) allows.
template <int NW, typename TO>
__device__ __forceinline__ void win_store_words(TO* p, const uint32_t (&w)[NW], int align)
{
    if (NW % 4 == 0 && align >= 16) {
        #pragma unroll
        for (int q = 0; q < NW / 4; ++q)
            reinterpret_cast<uint4*>(p)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else if (NW % 2 == 0 && align >= 8) {
        #pragma unroll
        for (int q = 0; q < NW / 2; ++q) reinterpret_cast<uint2*>(p)[q] = make_uint2(w[2 * q], w[2 * q + 1]);
    } else if (align >= 4) {
        #pragma unroll
        for (int q = 0; q < NW; ++q) reinterpret_cast<uint32_t*>(p)[q] = w[q];
    } else {
        #pragma unroll
        for (int q = 0; q < NW; ++q) {
            reinterpret_cast<uint16_t*>(p)[2 * q] = (uint16_t)w[q];
            reinterpret_cast<uint16_t*>(p)[2 * q + 1] = (uint16_t)(w[q] >> 16);
        }
    }
}

// X2: the first n elements of a run, one by one (the strip's ragged end).
template <int C, typename T>
__device__ __forceinline__ void win_store_part(T* p, const float2 (&v)[WinShape<C, T, true>::NP][C], int n)
{
    using S = WinShape<C, T, true>;
    #pragma unroll
    for (int e = 0; e < S::E; ++e) {
        if (e < n) {
            const int k = e / C, c = e % C;
            const float x = (k & 1) ? v[k >> 1][c].y : v[k >> 1][c].x;
            if constexpr (sizeof(T) == 1) p[e] = (uint8_t)win_u8(x);
            else Store<T>::put(p + e, x);
        }
    }
}

// General form: the C channels of one pixel at p (16-byte aligned rows allow
// one store per pixel when C * sizeof(T) is 4, 8 or 16 bytes).
template <int C, typename T>
__device__ __forceinline__ void win_store_px(T* p, const float (&x)[C], bool vec)
{
    constexpr int PB = C * (int)sizeof(T);
    if constexpr (sizeof(T) == 1 && (C == 4 || C == 2)) {
        if (vec) {
            if constexpr (C == 4)
                *reinterpret_cast<uint32_t*>(p) =
                    __byte_perm(__byte_perm(win_u8(x[0]), win_u8(x[1]), 0x0040), __byte_perm(win_u8(x[2]), win_u8(x[3]), 0x0040),
                                0x5410);
            else
                *reinterpret_cast<uint16_t*>(p) = (uint16_t)__byte_perm(win_u8(x[0]), win_u8(x[1]), 0x0040);
            return;
        }
    } else if constexpr (sizeof(T) == 2 && (C == 2 || C == 4)) {
        if (vec) {
            uint32_t w[C / 2];
            #pragma unroll
            for (int q = 0; q < C / 2; ++q) {
                if constexpr (std::is_same<T, __half>::value) {
                    const __half2 h = __floats2half2_rn(x[2 * q], x[2 * q + 1]);
                    w[q] = *reinterpret_cast<const uint32_t*>(&h);
                } else {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
                    w[q] = *reinterpret_cast<const uint32_t*>(&h);
                }
            }
            if constexpr (C == 2) *reinterpret_cast<uint32_t*>(p) = w[0];
            else *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
            return;
        }
    } else if constexpr (sizeof(T) == 4 && (C == 2 || C == 4)) {
        if (vec) {
            if constexpr (C == 2) *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
            else *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
            return;
        }
    }
    (void)PB;
    #pragma unroll
    for (int c = 0; c < C; ++c) {
        if constexpr (sizeof(T) == 1) p[c] = (uint8_t)win_u8(x[c]);
        else Store<T>::put(p + c, x[c]);
    }
}

// General form, the work of one block: strip bx and band by of one plane
// (s, d point at the plane). Used by the single-image kernel and the batch's
// persistent window kernels. TM = TAP_POINT: the taps of Eqs. 1-5 (KT = 2
// bilinear, 4 bicubic); TM = TAP_AA: the antialias taps (RS_FLAG_ANTIALIAS:
// the kernel of cfg.aa_method stretched by the downscale factor, at most KT
// per axis, renormalised), with half the pixels per lane at KT = 8.
enum { TAP_POINT = 0, TAP_AA = 1 };

template <int C, typename T, int TM, int KT>
struct WinGen {
    static constexpr int P0 = WinShape<C, T, false>::P;
    static constexpr int P = (TM == TAP_AA && KT > 4) ? (P0 / 2 < 2 ? 2 : P0 / 2) : P0;
    static constexpr int SP = kWinThreads * P;
};

template <int KT, int C, typename T, typename TO = T, bool NORM = false, int TM = TAP_POINT>
__device__ __forceinline__ void win_body(const Geom& g, const T* __restrict__ s, TO* __restrict__ d, const WinCfg& cfg,
                                         int bx, int by, float* sm, unsigned int* fault, const NormOut& no = NormOut{})
{
    using S = WinGen<C, T, TM, KT>;
    constexpr int P = S::P, NP = P / 2, NT = kWinThreads;
    constexpr int ES = (int)sizeof(T);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Strip of output pixels: 128 P, or for antialias taps cfg.strip <= 128 P
    // (a narrower strip keeps a large downscale's footprint in shared memory;
    // the lanes past it idle in the arithmetic and still stage rows).
    const int sw_px = TM == TAP_AA ? cfg.strip : S::SP;
    const int j_lo = bx * sw_px;                     // first pixel of the strip
    const int j_hi = min(g.Wo, j_lo + sw_px) - 1;    // last pixel of the strip
    const int yb = by * cfg.band_h;
    const int ye = min(g.Ho, yb + cfg.band_h);
    const int nrows = ye - yb;

    // Footprint of the strip: source pixels [px_lo, px_hi], unclamped. The
    // raw copy of a row starts at element base = px_lo C; staged rows are
    // channel-planar (plane c, position x = pixel px_lo + x), cfg.swe floats
    // per row.
    auto first_col = [&](int j) {
        if constexpr (TM == TAP_AA) {
            int lo, hi;
            aa_range(j, g.W, g.Wo, cfg.aa_method, lo, hi);
            return lo;
        } else {
            return first_tap<KT>(j, g.W, g.Wo, g.coord);
        }
    };
    const int px_lo = first_col(j_lo);
    const int px_hi = first_col(j_hi) + KT - 1;
    const int npx = px_hi - px_lo + 1;
    const int base = px_lo * C;
    const int span = npx * C;
    const int sw = cfg.swe / C;                   // floats per plane
    const int per = (span * ES + 15) / 16 + 1;    // raw 16-byte blocks per row
    const int in_lo = max(0, -px_lo) * C;         // raw elements [in_lo, in_hi) are in the image
    const int in_hi = (min(px_hi, g.W - 1) + 1) * C - base;
    if (per * 16 > cfg.raw_row || nrows > cfg.band_cap || npx > sw) {
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);   // uniform over the block
        return;
    }

    const int R = cfg.chunk;
    float* SR = sm;                                                           // [R][swe]
    float2* RW = reinterpret_cast<float2*>(reinterpret_cast<char*>(sm) + cfg.tab_off);   // [band_cap][KT] (w, w)
    int* RF = reinterpret_cast<int*>(RW + (size_t)cfg.band_cap * KT);         // [band_cap] first taps
    int* NC = RF + cfg.band_cap;                                              // [pos_cap] rows per position
    unsigned char* RAW = reinterpret_cast<unsigned char*>(sm) + cfg.raw_off;  // [2][R][raw_row]

    // Positions of the band: source rows b_first .. b_last are first taps.
    for (int i = tid; i < nrows; i += NT) {
        float w[KT];
        if constexpr (TM == TAP_AA) aa_taps<KT>(yb + i, g.H, g.Ho, cfg.aa_method, g.a, RF[i], w, fault);
        else RF[i] = taps<KT>(yb + i, g.H, g.Ho, g.coord, g.a, w);
        #pragma unroll
        for (int q = 0; q < KT; ++q) RW[i * KT + q] = make_float2(w[q], w[q]);
    }
    for (int q = tid; q < cfg.pos_cap; q += NT) NC[q] = 0;
    __syncthreads();   // row taps visible, NC cleared
    const int b_first = RF[0];
    const int b_last = RF[nrows - 1];
    if (b_last - b_first + 1 > cfg.pos_cap) {   // uniform; the host bounds the positions
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    for (int i0 = tid; i0 < nrows; i0 += NT) {   // rows per position (runs of equal first taps)
        if (i0 == 0 || RF[i0] != RF[i0 - 1]) {
            int len = 1;
            while (i0 + len < nrows && RF[i0 + len] == RF[i0]) ++len;
            NC[RF[i0] - b_first] = len;
        }
    }

    // ---- this lane's pixels jm = j0 + 32 m and their column taps ----
    const int j0 = j_lo + warp * 32 * P + lane;
    int off[P];          // planar position of each pixel's first tap
    bool valid[P];
    float2 wp[NP][KT];   // (weight of pixel 2p, weight of pixel 2p + 1) per tap
    #pragma unroll
    for (int p = 0; p < NP; ++p) {
        float w0[KT], w1[KT];
        #pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * p + h;
            const int j = j0 + 32 * m;
            float* w = h ? w1 : w0;
            valid[m] = j <= j_hi;
            if (valid[m]) {
                if constexpr (TM == TAP_AA) {
                    int lo;
                    aa_taps<KT>(j, g.W, g.Wo, cfg.aa_method, g.a, lo, w, fault);
                    off[m] = lo - px_lo;
                } else {
                    off[m] = taps<KT>(j, g.W, g.Wo, g.coord, g.a, w) - px_lo;
                }
            } else {
                off[m] = 0;
                #pragma unroll
                for (int q = 0; q < KT; ++q) w[q] = 0.0f;
            }
        }
        #pragma unroll
        for (int q = 0; q < KT; ++q) wp[p][q] = make_float2(w0[q], w1[q]);
    }

    // ---- staging ----
    const uintptr_t plane_lo = reinterpret_cast<uintptr_t>(s);
    const uintptr_t plane_hi = reinterpret_cast<uintptr_t>(s + (int64_t)(g.H - 1) * g.src_pitch + (int64_t)g.W * C);
    const uint32_t umul = 0xFFFFFFFFu / (uint32_t)per + 1u;
    auto row_ptr = [&](int r) -> const T* { return s + (int64_t)clampi(r, g.H) * g.src_pitch + base; };
    const int r_first = b_first, r_end = b_last + KT;   // source rows [r_first, r_end)
    auto chunk_rows = [&](int c) { return max(0, min(R, r_end - (r_first + c * R))); };
    // cp.async of the aligned blocks around rows of chunk c into raw slot c & 1
    auto issue = [&](int c) {
        const int r0 = r_first + c * R, nn = chunk_rows(c);
        unsigned char* rb = RAW + (size_t)(c & 1) * R * cfg.raw_row;
        for (int u = tid; u < nn * per; u += NT) {
            const int k = (int)__umulhi((uint32_t)u, umul), w = u - k * per;
            const T* rp = row_ptr(r0 + k);
            const uintptr_t ra = reinterpret_cast<uintptr_t>(rp);
            const uintptr_t blk = (ra & ~(uintptr_t)15) + 16 * (uintptr_t)w;
            unsigned char* dst = rb + k * cfg.raw_row + w * 16;
            if (blk >= plane_lo && blk + 16 <= plane_hi) {
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(reinterpret_cast<const void*>(blk))
                             : "memory");
            } else {
                // a block reaching outside the plane: only its in-image elements
                const int phase = (int)(ra & 15);
                const int e_lo = max(in_lo, (16 * w - phase + ES - 1) / ES);
                const int e_hi = min(in_hi, (16 * w + 16 - phase) / ES);
                for (int e = e_lo; e < e_hi; ++e) *reinterpret_cast<T*>(rb + k * cfg.raw_row + phase + e * ES) = rp[e];
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // raw slot -> channel-planar FP32 rows, one warp per row. Groups of 4
    // in-image pixels: one lane reads their C * sizeof(T) words (one funnel
    // shift realigns them), widens them and writes 4 floats to each plane.
    // The other pixels (edge pads, a partial last group) one per lane; an
    // out-of-image pixel reads the edge pixel (always in the footprint).
    const int xin_lo = max(0, -px_lo), xin_hi = min(npx, g.W - px_lo);   // in-image staged pixels
    const int g_lo = (xin_lo + 3) >> 2, g_hi = max(g_lo, xin_hi >> 2);   // whole in-image groups
    const int x_lo4 = min(4 * g_lo, npx), x_hi4 = max(4 * g_hi, x_lo4);
    auto convert = [&](int c) {
        const int r0 = r_first + c * R, nn = chunk_rows(c);
        const unsigned char* rbase = RAW + (size_t)(c & 1) * R * cfg.raw_row;
        for (int k = warp; k < nn; k += kWinWarps) {
            const int phase = (int)(reinterpret_cast<uintptr_t>(row_ptr(r0 + k)) & 15);
            const unsigned char* rrow = rbase + k * cfg.raw_row;
            float* dr = SR + k * cfg.swe;
            constexpr int GW = C * ES;   // words of a group of 4 pixels
            const uint32_t* W = reinterpret_cast<const uint32_t*>(rrow) + (phase >> 2);
            const int sh = 8 * (phase & 3);
            for (int q = g_lo + lane; q < g_hi; q += 32) {
                uint32_t x[GW + 1], y[GW];
                #pragma unroll
                for (int t = 0; t < GW + 1; ++t) x[t] = (ES < 4 || t < GW) ? W[q * GW + t] : 0u;
                #pragma unroll
                for (int t = 0; t < GW; ++t) y[t] = ES == 4 ? x[t] : __funnelshift_r(x[t], x[t + 1], sh);
                #pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    float f[4];
                    #pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int e = i * C + ch;   // element of the group
                        if constexpr (ES == 1)
                            f[i] = __int_as_float(__byte_perm(y[e >> 2], 0x4B000000u, 0x7650 + (e & 3))) - 8388608.0f;
                        else if constexpr (ES == 2) {
                            const uint32_t h16 = (y[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                            if constexpr (std::is_same<T, __half>::value) f[i] = __half2float(__ushort_as_half((unsigned short)h16));
                            else f[i] = __uint_as_float(h16 << 16);
                        } else
                            f[i] = __uint_as_float(y[e]);
                    }
                    *reinterpret_cast<float4*>(dr + ch * sw + 4 * q) = make_float4(f[0], f[1], f[2], f[3]);
                }
            }
            const T* rr = reinterpret_cast<const T*>(rrow + phase);   // element e at rr[e]
            const int nedge = x_lo4 + (npx - x_hi4);
            for (int t = lane; t < nedge; t += 32) {
                const int x = t < x_lo4 ? t : x_hi4 + (t - x_lo4);
                const int xs = min(max(px_lo + x, 0), g.W - 1) - px_lo;
                #pragma unroll
                for (int ch = 0; ch < C; ++ch) dr[ch * sw + x] = win_widen(rr[xs * C + ch]);
            }
        }
    };

    // ---- horizontal pass of one staged row: h[p][c] = (pixel 2p, pixel 2p + 1) ----
    auto hrow = [&](const float* Sr, float2 (&h)[NP][C]) {
        #pragma unroll
        for (int p = 0; p < NP; ++p)
            #pragma unroll
            for (int c = 0; c < C; ++c) h[p][c] = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int q = 0; q < KT; ++q)
            #pragma unroll
            for (int p = 0; p < NP; ++p)
                #pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float* pl = Sr + c * sw;
                    h[p][c] = __ffma2_rn(wp[p][q], make_float2(pl[off[2 * p] + q], pl[off[2 * p + 1] + q]), h[p][c]);
                }
    };

    // ---- output: one pixel's channels per store where the row allows it;
    // the fused pre-process: channel c normalised into its own plane ----
    const int pitch32 = (int)g.dst_pitch;   // the host bounds band_cap * pitch < 2^31
    constexpr int EO = (int)sizeof(TO);
    TO* const dband = d + (int64_t)yb * g.dst_pitch + (int64_t)j0 * (NORM ? 1 : C);
    constexpr int PB = C * ES;
    constexpr bool can_vec = !NORM && (PB == 4 || PB == 8 || PB == 16 || (PB == 2 && ES == 1));
    const bool vec0 = can_vec && (reinterpret_cast<uintptr_t>(dband) % PB) == 0;
    const bool vec_all = ((g.dst_pitch * EO) % PB) == 0;   // every row keeps row 0's alignment
    // (every pixel of the lane valid: one straight-line run of stores)
    const bool all_valid = valid[P - 1];
    auto put_px = [&](TO* p, int m, const float2 (&v)[NP][C], bool vec) {
        float x[C];
        #pragma unroll
        for (int c = 0; c < C; ++c) x[c] = (m & 1) ? v[m >> 1][c].y : v[m >> 1][c].x;
        if constexpr (NORM) {
            #pragma unroll
            for (int c = 0; c < C; ++c) Store<TO>::put(p + c * no.c_stride + 32 * m, fmaf(x[c], no.scale[c], no.bias[c]));
        } else {
            win_store_px<C, T>(p + 32 * m * C, x, vec);
        }
    };
    auto put = [&](int row, const float2 (&v)[NP][C]) {
        TO* p = dband + row * pitch32;
        const bool vec = can_vec && (vec_all ? vec0 : (reinterpret_cast<uintptr_t>(p) % PB) == 0);
        if (all_valid) {
            #pragma unroll
            for (int m = 0; m < P; ++m) put_px(p, m, v, vec);
        } else {
            #pragma unroll
            for (int m = 0; m < P; ++m)
                if (valid[m]) put_px(p, m, v, vec);
        }
    };

    // window: win[x][p][c] holds source row b + x at position b (slots rotate)
    float2 win[KT][NP][C];
    auto blend = [&](const float2* wrow, const int* slot, float2 (&v)[NP][C]) {
        // the row's (w, w) pairs two per 16-byte load (the table and its rows
        // are 16-byte aligned)
        float2 wr[KT];
        #pragma unroll
        for (int q = 0; q < KT; q += 2) {
            const float4 w4 = *reinterpret_cast<const float4*>(wrow + q);
            wr[q] = make_float2(w4.x, w4.y);
            wr[q + 1] = make_float2(w4.z, w4.w);
        }
        #pragma unroll
        for (int p = 0; p < NP; ++p)
            #pragma unroll
            for (int c = 0; c < C; ++c) v[p][c] = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float2 w2 = wr[q];
            #pragma unroll
            for (int p = 0; p < NP; ++p)
                #pragma unroll
                for (int c = 0; c < C; ++c) v[p][c] = __ffma2_rn(w2, win[slot[q]][p][c], v[p][c]);
        }
    };

    // ---- prologue: chunks 0 and 1 in flight, chunk 0 staged ----
    int cidx = 0, chunk_lo = r_first, nn = chunk_rows(0);
    issue(0);
    issue(1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    convert(0);
    __syncthreads();
    issue(2);

    int i = 0;          // next output row of the band
    int b = b_first;    // current position
    #pragma unroll
    for (int x = 0; x < KT - 1; ++x) hrow(SR + x * cfg.swe, win[x]);
    int r = b_first + KT - 1;   // next source row to interpolate

    while (b <= b_last) {
        #pragma unroll
        for (int u = 0; u < KT; ++u) {
            if (b <= b_last) {
                // Source row r = b + KT - 1 enters the staged chunk only at u == 1
                // (chunks are whole groups of KT rows from r_first).
                if (u == 1 && r >= chunk_lo + nn) {
                    ++cidx;
                    chunk_lo = r_first + cidx * R;
                    nn = chunk_rows(cidx);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                    __syncthreads();   // copies of chunk cidx landed; the FP32 rows are read
                    convert(cidx);
                    __syncthreads();   // chunk cidx staged; its raw slot is free
                    issue(cidx + 2);
                }
                const int ns = (u + KT - 1) % KT;   // the newest row's slot
                hrow(SR + (r - chunk_lo) * cfg.swe, win[ns]);
                ++r;
                int slot[KT];
                #pragma unroll
                for (int x = 0; x < KT; ++x) slot[x] = (u + x) % KT;
                // the rows of this position, two at a time (independent FMA chains)
                const int nb = NC[b - b_first];
                int k = 0;
                for (; k + 1 < nb; k += 2) {
                    float2 v0[NP][C], v1[NP][C];
                    blend(RW + (size_t)(i + k) * KT, slot, v0);
                    blend(RW + (size_t)(i + k + 1) * KT, slot, v1);
                    put(i + k, v0);
                    put(i + k + 1, v1);
                }
                if (k < nb) {
                    float2 v0[NP][C];
                    blend(RW + (size_t)(i + k) * KT, slot, v0);
                    put(i + k, v0);
                }
                i += nb;
                ++b;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // nothing in flight when the block moves on
}

// Exact-x2 form (the asymmetric map at exactly x2 on both axes), the work of
// one block: strip bx and band by of one plane. Each thread widens its own
// footprint (P/2 + KT - 1 source pixels) straight from the raw copy of a
// source row: no FP32 staging, one barrier per chunk, a three-slot raw ring
// with two chunks in flight. Out-of-image footprint pixels (strips at the
// image's left and right edges only) are written into the raw rows as copies
// of the edge pixel once a chunk has landed.
template <int KT, int C, typename T, typename TO = T, bool NORM = false>
__device__ __forceinline__ void win_body_x2(const Geom& g, const T* __restrict__ s, TO* __restrict__ d,
                                            const WinCfg& cfg, int bx, int by, float* sm, unsigned int* fault,
                                            const NormOut& no = NormOut{})
{
    using S = WinShape<C, T, true>;
    constexpr int P = S::P, NP = S::NP, NT = kWinThreads;
    constexpr int ES = (int)sizeof(T);
    constexpr int HK = KT / 2 - 1;              // footprint pixels left of a thread's first source pixel
    constexpr int FPL = (NP + KT - 1) * C;      // footprint elements of a thread
    constexpr int NF = (FPL * ES + 3) / 4;      // footprint words (after the byte shift)
    constexpr int NR = ES == 4 ? NF : NF + 1;   // words read
    const int tid = threadIdx.x;

    const int j_lo = bx * S::SP;
    const int j_hi = min(g.Wo, j_lo + S::SP) - 1;
    const int yb = by * cfg.band_h;
    const int ye = min(g.Ho, yb + cfg.band_h);
    const int nrows = ye - yb;
    // Footprint of the strip: source pixels [px_lo, px_hi] (first taps j / 2 - HK);
    // the raw copy of a row starts at element base = px_lo C.
    const int px_lo = j_lo / 2 - HK;
    const int px_hi = j_hi / 2 - HK + KT - 1;
    const int base = px_lo * C;
    const int span = (px_hi - px_lo + 1) * C;
    const int per = (span * ES + 15) / 16 + 1;    // raw 16-byte blocks copied per row
    const int in_lo = max(0, -px_lo) * C;         // raw elements [in_lo, in_hi) are in the image
    const int in_hi = (min(px_hi, g.W - 1) + 1) * C - base;
    // thread t reads words of bytes [0, 16 + t HALF ES + 4 NR) of a raw row
    if (per * 16 > cfg.raw_row || 16 + (NT - 1) * S::HALF * ES + 4 * NR > cfg.raw_row || ((yb | nrows) & 1)) {
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);   // uniform over the block
        return;
    }
    const int R = cfg.chunk;
    unsigned char* RAW = reinterpret_cast<unsigned char*>(sm);   // [3][R][raw_row]
    const int b_first = yb / 2 - HK, b_last = (ye - 1) / 2 - HK;   // positions (first taps) of the band
    const bool edge = px_lo < 0 || px_hi >= g.W;                    // uniform over the block

    const int j0 = j_lo + tid * P;                      // this thread's run j0 .. j0 + P - 1
    const int nact = max(0, min(P, j_hi - j0 + 1));     // pixels of the run inside the strip
    float wx2[KT];                                      // the t = 1/2 weights
    tap_weights<KT>(0.5f, g.a, wx2);
    float2 wy2[KT];
    #pragma unroll
    for (int q = 0; q < KT; ++q) wy2[q] = make_float2(wx2[q], wx2[q]);

    // ---- staging ----
    const uintptr_t plane_lo = reinterpret_cast<uintptr_t>(s);
    const uintptr_t plane_hi = reinterpret_cast<uintptr_t>(s + (int64_t)(g.H - 1) * g.src_pitch + (int64_t)g.W * C);
    const uint32_t umul = 0xFFFFFFFFu / (uint32_t)per + 1u;
    auto row_ptr = [&](int r) -> const T* { return s + (int64_t)clampi(r, g.H) * g.src_pitch + base; };
    const int r_first = b_first, r_end = b_last + KT;   // source rows [r_first, r_end)
    auto chunk_rows = [&](int c) { return max(0, min(R, r_end - (r_first + c * R))); };
    auto slot_ptr = [&](int c) { return RAW + (size_t)(c % 3) * R * cfg.raw_row; };
    auto issue = [&](int c) {
        const int r0 = r_first + c * R, nn = chunk_rows(c);
        unsigned char* rb = slot_ptr(c);
        for (int u = tid; u < nn * per; u += NT) {
            const int k = (int)__umulhi((uint32_t)u, umul), w = u - k * per;
            const T* rp = row_ptr(r0 + k);
            const uintptr_t ra = reinterpret_cast<uintptr_t>(rp);
            const uintptr_t blk = (ra & ~(uintptr_t)15) + 16 * (uintptr_t)w;
            unsigned char* dst = rb + k * cfg.raw_row + w * 16;
            if (blk >= plane_lo && blk + 16 <= plane_hi) {
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(reinterpret_cast<const void*>(blk))
                             : "memory");
            } else {
                const int phase = (int)(ra & 15);
                const int e_lo = max(in_lo, (16 * w - phase + ES - 1) / ES);
                const int e_hi = min(in_hi, (16 * w + 16 - phase) / ES);
                for (int e = e_lo; e < e_hi; ++e) *reinterpret_cast<T*>(rb + k * cfg.raw_row + phase + e * ES) = rp[e];
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // edge pads of a landed chunk: positions outside [in_lo, in_hi) take the edge pixel
    auto padfix = [&](int c) {
        const int r0 = r_first + c * R, nn = chunk_rows(c);
        unsigned char* rb = slot_ptr(c);
        const int npad = in_lo + (span - in_hi);
        for (int u = tid; u < nn * npad; u += NT) {
            const int k = u / npad, q0 = u - k * npad;
            const int q = q0 < in_lo ? q0 : in_hi + (q0 - in_lo);
            const int src = (q < in_lo ? in_lo : in_hi - C) + q % C;
            T* rr = reinterpret_cast<T*>(rb + k * cfg.raw_row + (int)(reinterpret_cast<uintptr_t>(row_ptr(r0 + k)) & 15));
            rr[q] = rr[src];
        }
    };

    // ---- horizontal pass of source row r (in the current chunk) ----
    // h[p][c] = (pixel 2p: the sample itself, pixel 2p + 1: the t = 1/2 blend)
    auto hrow = [&](const unsigned char* rrow, int phase, float2 (&h)[NP][C]) {
        const int o = phase + tid * (S::HALF * ES);   // byte of this thread's first footprint element
        const uint32_t* W = reinterpret_cast<const uint32_t*>(rrow) + (o >> 2);
        uint32_t x[NR];
        #pragma unroll
        for (int k = 0; k < NR; ++k) x[k] = W[k];
        uint32_t y[NF];
        if constexpr (ES == 4) {
            #pragma unroll
            for (int k = 0; k < NF; ++k) y[k] = x[k];
        } else {
            const int sh = 8 * (o & 3);
            #pragma unroll
            for (int k = 0; k < NF; ++k) y[k] = __funnelshift_r(x[k], x[k + 1], sh);
        }
        float F[FPL + 2 * NF + 2];
        if constexpr (ES == 1) {
            const float2 M = make_float2(-8388608.0f, -8388608.0f);
            #pragma unroll
            for (int e = 0; e < FPL; e += 2) {
                const float2 f = __fadd2_rn(make_float2(__int_as_float(__byte_perm(y[e >> 2], 0x4B000000u, 0x7650 + (e & 3))),
                                                        __int_as_float(__byte_perm(y[(e + 1) >> 2], 0x4B000000u,
                                                                                   0x7650 + ((e + 1) & 3)))), M);
                F[e] = f.x;
                F[e + 1] = f.y;
            }
        } else if constexpr (ES == 2) {
            #pragma unroll
            for (int k = 0; k < NF; ++k) {
                float2 f;
                if constexpr (std::is_same<T, __half>::value) f = __half22float2(*reinterpret_cast<const __half2*>(&y[k]));
                else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&y[k]));
                F[2 * k] = f.x;
                F[2 * k + 1] = f.y;
            }
        } else {
            #pragma unroll
            for (int k = 0; k < NF; ++k) F[k] = __uint_as_float(y[k]);
        }
        #pragma unroll
        for (int p = 0; p < NP; ++p) {
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                float od = 0.0f;
                #pragma unroll
                for (int q = 0; q < KT; ++q) od = fmaf(wx2[q], F[(p + q) * C + c], od);
                h[p][c] = make_float2(F[(p + HK) * C + c], od);
            }
        }
    };

    // ---- output: the run as 4-, 8- or 16-byte stores; the fused
    // pre-process: each channel's P values normalised into its own plane ----
    const int pitch32 = (int)g.dst_pitch;   // the host bounds band_cap * pitch < 2^31
    constexpr int EO = (int)sizeof(TO);
    TO* const dband = d + (int64_t)yb * g.dst_pitch + (int64_t)j0 * (NORM ? 1 : C);
    const bool same_align = ((g.dst_pitch * EO) & 15) == 0 && (!NORM || ((no.c_stride * EO) & 15) == 0);
    auto align_of = [&](const TO* p) -> int {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        return (a & 15) == 0 ? 16 : (a & 7) == 0 ? 8 : (a & 3) == 0 ? 4 : (a & 1) == 0 ? 2 : 1;
    };
    const int align0 = align_of(dband);
    auto put = [&](int row, const float2 (&v)[NP][C]) {
        TO* p = dband + row * pitch32;
        if constexpr (NORM) {
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                TO* pc = p + c * no.c_stride;
                float y[P];
                #pragma unroll
                for (int k = 0; k < P; ++k) y[k] = fmaf((k & 1) ? v[k >> 1][c].y : v[k >> 1][c].x, no.scale[c], no.bias[c]);
                if (nact == P && (P * EO) % 4 == 0) {
                    uint32_t w[P * EO / 4];
                    win_pack_plane<P, TO>(y, w);
                    win_store_words<P * EO / 4>(pc, w, same_align ? align0 : align_of(pc));
                } else {
                    #pragma unroll
                    for (int k = 0; k < P; ++k)
                        if (k < nact) Store<TO>::put(pc + k, y[k]);
                }
            }
        } else {
            if (nact == P) {
                uint32_t w[S::NW];
                win_pack<C, T>(v, w);
                win_store_run<C, T>(p, w, same_align ? align0 : align_of(p));
            } else if (nact > 0) {
                win_store_part<C, T>(p, v, nact * C);
            }
        }
    };

    float2 win[KT][NP][C];   // win[x]: source row b + x at position b (slots rotate)
    auto blend = [&](const int* slot, float2 (&v)[NP][C]) {
        #pragma unroll
        for (int p = 0; p < NP; ++p)
            #pragma unroll
            for (int c = 0; c < C; ++c) v[p][c] = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int q = 0; q < KT; ++q)
            #pragma unroll
            for (int p = 0; p < NP; ++p)
                #pragma unroll
                for (int c = 0; c < C; ++c) v[p][c] = __ffma2_rn(wy2[q], win[slot[q]][p][c], v[p][c]);
    };

    // ---- prologue: chunks 0, 1, 2 in flight; chunk 0 landed ----
    int cidx = 0, chunk_lo = r_first, nn = chunk_rows(0);
    issue(0);
    issue(1);
    issue(2);
    asm volatile("cp.async.wait_group 2;" ::: "memory");
    __syncthreads();
    if (edge) {
        padfix(0);
        __syncthreads();
    }
    auto row_bytes = [&](int r) { return slot_ptr(cidx) + (r - chunk_lo) * cfg.raw_row; };
    auto row_phase = [&](int r) { return (int)(reinterpret_cast<uintptr_t>(row_ptr(r)) & 15); };
    #pragma unroll
    for (int x = 0; x < KT - 1; ++x) hrow(row_bytes(r_first + x), row_phase(r_first + x), win[x]);

    int i = 0;                  // next output row of the band
    int b = b_first;            // current position
    int r = b_first + KT - 1;   // next source row to interpolate
    while (b <= b_last) {
        #pragma unroll
        for (int u = 0; u < KT; ++u) {
            if (b <= b_last) {
                if (u == 1 && r >= chunk_lo + nn) {   // next chunk (chunks are whole groups of KT rows)
                    ++cidx;
                    chunk_lo = r_first + cidx * R;
                    nn = chunk_rows(cidx);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                    __syncthreads();   // chunk cidx landed; every thread is done with chunk cidx - 1
                    if (edge) {
                        padfix(cidx);
                        __syncthreads();
                    }
                    issue(cidx + 2);   // into the slot of chunk cidx - 1
                }
                hrow(row_bytes(r), row_phase(r), win[(u + KT - 1) % KT]);
                ++r;
                int slot[KT];
                #pragma unroll
                for (int x = 0; x < KT; ++x) slot[x] = (u + x) % KT;
                // rows 2(b + HK) (t = 0: window row b + HK) and 2(b + HK) + 1 (t = 1/2)
                float2 v[NP][C];
                blend(slot, v);
                put(i, win[slot[HK]]);
                put(i + 1, v);
                i += 2;
                ++b;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // nothing in flight when the block moves on
}

}  // namespace rs
