// Antialiased resampling with more taps per axis than the register-window
// forms hold (RS_FLAG_ANTIALIAS at large downscales: bilinear below 1/4,
// bicubic below 1/2): the work of one block, shared by the single-image
// kernel (aa_wide.cu) and the batch (batched.cu).
//
// One block of 256 threads per output tile of kAwTW columns x TH rows of one
// plane. The tile's taps (any count up to the host's bound) go to shared
// memory; the source rows its y taps reach are copied, RG at a time, into
// shared memory as FP32 (coalesced along the row) and horizontally
// interpolated at the tile's columns into an FP32 buffer of footprint rows
// x tile columns; the tile's outputs are then blended from that buffer.
// Sums run over the taps in ascending order, x first, then y (the order of
// the window forms).
#pragma once

#include "rs_common.cuh"

namespace rs {

static constexpr int kAwTW = 32;   // output columns per tile
static constexpr int kAwNT = 256;  // threads per block

template <int C, typename T, typename TO, bool NORM>
__device__ __forceinline__ void aa_wide_body(const Geom& g, const T* __restrict__ s, TO* __restrict__ d,
                                             const AaWideCfg& cfg, int bx, int by, float* sm, unsigned int* fault,
                                             const NormOut& no)
{
    const int tid = threadIdx.x;
    const int j0 = bx * kAwTW, i0 = by * cfg.TH;
    const int nj = min(kAwTW, g.Wo - j0), ni = min(cfg.TH, g.Ho - i0);
    constexpr int TWC = kAwTW * C;

    float* WX = sm;                                       // [kAwTW][KX]
    float* WY = WX + kAwTW * cfg.KX;                      // [TH][KY]
    int* LX = reinterpret_cast<int*>(WY + cfg.TH * cfg.KY);   // [kAwTW] first x tap - px_lo
    int* CX = LX + kAwTW;                                 // [kAwTW] x tap counts
    int* LY = CX + kAwTW;                                 // [TH] first y tap - r_lo
    int* CY = LY + cfg.TH;                                // [TH] y tap counts
    float* S = sm + cfg.s_off;                            // [RG][fw C] staged source rows
    float* HB = S + (size_t)cfg.RG * cfg.fw * C;          // [nr][kAwTW C] horizontal results

    int px_lo, px_hi, r_lo, r_hi, t0, t1;
    aa_range(j0, g.W, g.Wo, cfg.method, px_lo, t0);
    aa_range(j0 + nj - 1, g.W, g.Wo, cfg.method, t1, px_hi);   // exclusive
    aa_range(i0, g.H, g.Ho, cfg.method, r_lo, t0);
    aa_range(i0 + ni - 1, g.H, g.Ho, cfg.method, t1, r_hi);
    const int npx = px_hi - px_lo, nr = r_hi - r_lo;
    if (npx > cfg.fw || nr > cfg.nr || npx < 1 || nr < 1) {   // uniform; the host bounds both
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    if (tid < kAwTW) {
        int lo = 0, cnt = 0;
        if (tid < nj) cnt = aa_taps_n(j0 + tid, g.W, g.Wo, cfg.method, g.a, cfg.KX, lo, WX + tid * cfg.KX, fault);
        LX[tid] = tid < nj ? lo - px_lo : 0;
        CX[tid] = cnt;
    } else if (tid < kAwTW + ni) {
        const int i = tid - kAwTW;
        int lo = 0;
        CY[i] = aa_taps_n(i0 + i, g.H, g.Ho, cfg.method, g.a, cfg.KY, lo, WY + i * cfg.KY, fault);
        LY[i] = lo - r_lo;
    }
    __syncthreads();

    // horizontal pass over the footprint rows, RG at a time
    const int rowe = npx * C;   // staged elements per row
    for (int rg = 0; rg < nr; rg += cfg.RG) {
        const int nn = min(cfg.RG, nr - rg);
        for (int e = tid; e < nn * rowe; e += kAwNT) {
            const int r = e / rowe, x = e - r * rowe;
            S[r * cfg.fw * C + x] = Store<T>::load(s + (int64_t)(r_lo + rg + r) * g.src_pitch + (int64_t)px_lo * C + x);
        }
        __syncthreads();
        for (int e = tid; e < nn * TWC; e += kAwNT) {
            const int r = e / TWC, jc = e - r * TWC, j = jc / C, c = jc - j * C;
            const float* row = S + r * cfg.fw * C + LX[j] * C + c;
            const float* w = WX + j * cfg.KX;
            float acc = 0.0f;
            for (int k = 0; k < CX[j]; ++k) acc = fmaf(w[k], row[k * C], acc);
            HB[(size_t)(rg + r) * TWC + jc] = acc;
        }
        __syncthreads();
    }

    // vertical pass and store
    for (int e = tid; e < ni * TWC; e += kAwNT) {
        const int i = e / TWC, jc = e - i * TWC, j = jc / C, c = jc - j * C;
        if (j >= nj) continue;
        const float* col = HB + (size_t)LY[i] * TWC + jc;
        const float* w = WY + i * cfg.KY;
        float acc = 0.0f;
        for (int k = 0; k < CY[i]; ++k) acc = fmaf(w[k], col[(size_t)k * TWC], acc);
        const int64_t row = (int64_t)(i0 + i) * g.dst_pitch;
        if constexpr (NORM) Store<TO>::put(d + c * no.c_stride + row + j0 + j, fmaf(acc, no.scale[c], no.bias[c]));
        else Store<TO>::put(d + row + (int64_t)(j0 + j) * C + c, acc);
    }
}

}  // namespace rs
