// Antialiased resampling of vertical downscales, vertical pass first, with
// the source rows streamed once through a shared-memory copy ring and the
// vertical sums kept in registers (RS_FLAG_ANTIALIAS where the output rows
// are no more than the source rows and the window forms do not apply).
//
// One block of 256 threads per output tile of TW columns x TH rows of one
// plane. The tile's source footprint (the source columns its TW outputs' x
// taps reach, times the channels: at most 1024 elements, 4 per thread) is
// walked once, top to bottom: rows are copied with 16-byte cp.async (the
// aligned blocks around each row) into a three-slot ring of R-row chunks,
// two chunks ahead. Thread t owns footprint elements 4t .. 4t + 3 and adds
// each row into the register slot of every tile row whose y taps include
// that row: tile row i uses slot i mod NA, and the host checks that a slot's
// next row starts at or below the previous one's last tap. A per-row table
// holds the row's weight in each slot and the tile rows (if any) whose last
// tap it is. When a tile row is complete its slot goes to one of NB = 8
// shared-memory row buffers; after every NB rows (and after the last) the
// block blends those rows' outputs with their x taps and stores them, between
// two barriers. Sums run over the taps
// in ascending order, y first, then x.
#pragma once

#include "rs_common.cuh"

namespace rs {

static constexpr int kVsNT = 256;  // threads per block
static constexpr int kVsE = 4;     // footprint elements per thread
static constexpr int kVsNB = 8;    // finished-row buffers (rows blended per batch)

__device__ __forceinline__ float vs_widen(uint8_t v) { return __uint_as_float(0x4B000000u | v) - 8388608.0f; }
__device__ __forceinline__ float vs_widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float vs_widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float vs_widen(float v) { return v; }

template <int C, typename T, typename TO, bool NORM, int NA>
__device__ __forceinline__ void aa_vs_body(const Geom& g, const T* __restrict__ s, TO* __restrict__ d,
                                           const AaVsCfg& cfg, int bx, int by, float* sm, unsigned int* fault,
                                           const NormOut& no)
{
    constexpr int E = kVsE, NT = kVsNT;
    constexpr int ES = (int)sizeof(T);
    const int tid = threadIdx.x;
    const int TW = cfg.TW, R = cfg.chunk;
    const int j0 = bx * TW, i0 = by * cfg.TH;
    const int nj = min(TW, g.Wo - j0), ni = min(cfg.TH, g.Ho - i0);
    const int m = cfg.method;

    int px_lo, px_hi, r_lo, r_hi, t0, t1;
    aa_range(j0, g.W, g.Wo, m, px_lo, t0);
    aa_range(j0 + nj - 1, g.W, g.Wo, m, t1, px_hi);   // exclusive
    aa_range(i0, g.H, g.Ho, m, r_lo, t0);
    aa_range(i0 + ni - 1, g.H, g.Ho, m, t1, r_hi);
    const int npx = px_hi - px_lo, nr = r_hi - r_lo, ne = npx * C;
    const int per = (ne * ES + 15) / 16 + 1;   // 16-byte blocks around a row's footprint
    if (ne > cfg.ve || ne > NT * E || nr > cfg.nr || (per + 1) * 16 > cfg.raw_row || npx < 1 || nr < 1) {
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);   // uniform; bounded by the host
        return;
    }
    unsigned char* RAW = reinterpret_cast<unsigned char*>(sm);                  // [3][R][raw_row]
    float* V = reinterpret_cast<float*>(RAW + (size_t)3 * R * cfg.raw_row);     // [NB][ve] finished rows
    float* WX = V + kVsNB * (size_t)cfg.ve;                                      // [TW][KX]
    float* YW = WX + (size_t)TW * cfg.KX;                                        // [nr][NA] row weight per slot
    int* LX = reinterpret_cast<int*>(YW + (size_t)cfg.nr * NA);                  // [TW] first x tap - px_lo
    int* CX = LX + TW;                                                           // [TW] x tap counts
    int* FIN = CX + TW;                                                          // [nr] first tile row ending here
    int* NFIN = FIN + cfg.nr;                                                    // [nr] tile rows ending here

    // ---- copies: the aligned 16-byte blocks around rows of chunk c into slot c % 3 ----
    const uintptr_t plane_lo = reinterpret_cast<uintptr_t>(s);
    const uintptr_t plane_hi = reinterpret_cast<uintptr_t>(s + (int64_t)(g.H - 1) * g.src_pitch + (int64_t)g.W * C);
    const uint32_t umul = 0xFFFFFFFFu / (uint32_t)per + 1u;
    auto row_ptr = [&](int y) -> const T* { return s + (int64_t)(r_lo + y) * g.src_pitch + (int64_t)px_lo * C; };
    const int nchunks = (nr + R - 1) / R;
    auto issue = [&](int c) {
        const int y0 = c * R, nn = max(0, min(R, nr - y0));
        unsigned char* rb = RAW + (size_t)(c % 3) * R * cfg.raw_row;
        for (int u = tid; u < nn * per; u += NT) {
            const int k = (int)__umulhi((uint32_t)u, umul), w = u - k * per;
            const T* rp = row_ptr(y0 + k);
            const uintptr_t ra = reinterpret_cast<uintptr_t>(rp);
            const uintptr_t blk = (ra & ~(uintptr_t)15) + 16 * (uintptr_t)w;
            unsigned char* dst = rb + k * cfg.raw_row + w * 16;
            if (blk >= plane_lo && blk + 16 <= plane_hi) {
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(reinterpret_cast<const void*>(blk))
                             : "memory");
            } else {
                // a block reaching outside the plane: only the footprint's elements in it
                const int phase = (int)(ra & 15);
                const int e_lo = max(0, (16 * w - phase + ES - 1) / ES);
                const int e_hi = min(ne, (16 * w + 16 - phase) / ES);
                for (int e = e_lo; e < e_hi; ++e) *reinterpret_cast<T*>(rb + k * cfg.raw_row + phase + e * ES) = rp[e];
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    issue(1);

    // ---- tap tables ----
    for (int e = tid; e < nr * NA; e += NT) YW[e] = 0.0f;
    for (int e = tid; e < nr; e += NT) NFIN[e] = 0;
    __syncthreads();
    for (int j = tid; j < TW; j += NT) {
        int lo = 0, cnt = 0;
        if (j < nj) cnt = aa_taps_n(j0 + j, g.W, g.Wo, m, g.a, cfg.KX, lo, WX + j * cfg.KX, fault);
        LX[j] = j < nj ? lo - px_lo : 0;
        CX[j] = cnt;
    }
    for (int i = tid; i < ni; i += NT) {
        // tile row i: its renormalised y taps into its slot's column
        int lo, hi;
        aa_range(i0 + i, g.H, g.Ho, m, lo, hi);
        const float inv2F = 1.0f / (2.0f * (float)max(g.H, g.Ho));
        const int64_t cj = (int64_t)(2 * (i0 + i) + 1) * g.H;
        float* col = YW + (size_t)(lo - r_lo) * NA + i % NA;
        float tot = 0.0f;
        for (int k = 0; k < hi - lo; ++k) {
            const float v = aa_kernel(lo + k, g.Ho, cj, inv2F, m, g.a);
            col[(size_t)k * NA] = v;
            tot += v;
        }
        const float inv = tot != 0.0f ? 1.0f / tot : 1.0f;
        for (int k = 0; k < hi - lo; ++k) col[(size_t)k * NA] *= inv;
        // one row ends on each row above the footprint's last; on the last
        // row end the tile's last row and, at the image's bottom, the rows
        // whose taps are cut there (consecutive, at most NA)
        if (hi < r_hi) {
            FIN[hi - 1 - r_lo] = i;
            NFIN[hi - 1 - r_lo] = 1;
        }
    }
    if (tid == 0) {
        int first = ni - 1;
        while (first > 0 && first > ni - NA) {
            int lo, hi;
            aa_range(i0 + first - 1, g.H, g.Ho, m, lo, hi);
            if (hi < r_hi) break;
            --first;
        }
        FIN[nr - 1] = first;
        NFIN[nr - 1] = ni - first;
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();   // tables and chunk 0 visible
    issue(2);

    // ---- vertical pass ----
    const int e0 = tid * E;
    float2 acc[NA][E / 2];   // element pairs (packed FP32x2 FMAs)
    #pragma unroll
    for (int q = 0; q < NA; ++q)
        #pragma unroll
        for (int k = 0; k < E / 2; ++k) acc[q][k] = make_float2(0.0f, 0.0f);
    // tile row f is complete: its slot into row buffer f % NB. A full batch
    // of NB rows (or the last rows) is then blended with the x taps and
    // stored, between two barriers.
    auto blend_rows = [&](int fa, int fb) {   // tile rows fa .. fb (at most NB)
        __syncthreads();   // the rows' buffers complete
        const int njc = nj * C;
        for (int e = tid; e < (fb - fa + 1) * njc; e += NT) {
            const int r = e / njc, jc = e - r * njc, f = fa + r;
            const int j = jc / C, c = jc - j * C;
            const float* row = V + (size_t)(f % kVsNB) * cfg.ve + LX[j] * C + c;
            const float* w = WX + j * cfg.KX;
            const int cnt = CX[j];
            float a2 = 0.0f;
            int k = 0;
            for (; k + 4 <= cnt; k += 4) {
                a2 = fmaf(w[k], row[k * C], a2);
                a2 = fmaf(w[k + 1], row[(k + 1) * C], a2);
                a2 = fmaf(w[k + 2], row[(k + 2) * C], a2);
                a2 = fmaf(w[k + 3], row[(k + 3) * C], a2);
            }
            for (; k < cnt; ++k) a2 = fmaf(w[k], row[k * C], a2);
            const int64_t orow = (int64_t)(i0 + f) * g.dst_pitch;
            if constexpr (NORM) Store<TO>::put(d + c * no.c_stride + orow + j0 + j, fmaf(a2, no.scale[c], no.bias[c]));
            else Store<TO>::put(d + orow + (int64_t)(j0 + j) * C + c, a2);
        }
        __syncthreads();   // the buffers free for the next batch
    };
    auto finish = [&](int f) {
        const int sl = f % NA;
        float* vr = V + (size_t)(f % kVsNB) * cfg.ve;
        #pragma unroll
        for (int q = 0; q < NA; ++q)
            if (q == sl) {
                if (e0 < ne)
                    *reinterpret_cast<float4*>(vr + e0) = make_float4(acc[q][0].x, acc[q][0].y, acc[q][1].x, acc[q][1].y);
                #pragma unroll
                for (int k = 0; k < E / 2; ++k) acc[q][k] = make_float2(0.0f, 0.0f);
            }
        if (f % kVsNB == kVsNB - 1) blend_rows(f - kVsNB + 1, f);   // uniform
    };
    for (int c = 0; c < nchunks; ++c) {
        if (c > 0) {
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncthreads();   // chunk c landed; chunk c - 1 no longer read
            issue(c + 2);
        }
        const int nn = min(R, nr - c * R);
        // this thread's elements of row k of the chunk: footprint element e
        // at byte (phase of the row) + e * ES of the raw row; the raw rows
        // hold a spare 16-byte block, so the 4 elements of the thread that
        // holds the footprint's end can be read whole (the ones past the end
        // are never stored)
        const unsigned char* rb = RAW + (size_t)(c % 3) * R * cfg.raw_row + e0 * ES;
        int phase = (int)(reinterpret_cast<uintptr_t>(row_ptr(c * R)) & 15);
        const int dphase = (int)((g.src_pitch * ES) & 15);
        for (int k = 0; k < nn; ++k) {
            const int y = c * R + k;
            float2 x01 = make_float2(0.0f, 0.0f), x23 = x01;
            if (e0 < ne) {
                const T* rr = reinterpret_cast<const T*>(rb + k * cfg.raw_row + phase);
                x01 = make_float2(vs_widen(rr[0]), vs_widen(rr[1]));
                x23 = make_float2(vs_widen(rr[2]), vs_widen(rr[3]));
            }
            phase = (phase + dphase) & 15;
            const float* wy = YW + y * NA;
            #pragma unroll
            for (int q = 0; q < NA; ++q) {
                const float w = wy[q];
                acc[q][0] = __ffma2_rn(make_float2(w, w), x01, acc[q][0]);
                acc[q][1] = __ffma2_rn(make_float2(w, w), x23, acc[q][1]);
            }
            const int nf = NFIN[y];
            for (int t = 0; t < nf; ++t) finish(FIN[y] + t);   // uniform
        }
    }
    if (ni % kVsNB) blend_rows(ni - ni % kVsNB, ni - 1);   // the last, partial batch
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // nothing in flight when the block ends
}

}  // namespace rs
