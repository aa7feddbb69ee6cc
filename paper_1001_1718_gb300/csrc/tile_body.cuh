// The per-tile work of the tiled forward kernel, shared by the single-image
// kernel (one tile per thread block) and the persistent batched kernel (a
// block walks a list of tiles of many images).
//
// A tile is cfg.tile_w output ELEMENTS (an output row holds Wo * C
// interleaved elements) by cfg.tile_h output rows of one plane:
//   1. row taps (Eqs. 1-4 on the y axis) go to shared memory; each thread
//      computes the column taps of its four output elements;
//   2. the tile's source footprint (rows and columns plus the tap halo,
//      clamped to the image: edge replicate) is staged in shared memory as
//      FP32;
//   3. horizontal pass: each staged source row is interpolated at the tile's
//      output columns into a second shared buffer;
//   4. vertical pass: each output row blends its taps' rows of that buffer
//      (Eq. 5 generalised to 1, 2 or 4 taps), rounds to the storage type and
//      stores four consecutive elements per thread.
// The separable order costs taps * (1/scale + 1) multiply-adds per output
// element at upscale instead of taps^2.
#pragma once

#include "rs_common.cuh"

namespace rs {

template <int KT, int C, typename T>
__device__ __forceinline__ void tile_body(const Geom& g, const T* __restrict__ s, T* __restrict__ d,
                                          const TileCfg& cfg, int bx, int by, float* sm,
                                          unsigned int* fault)
{
    const int TWE = cfg.tile_w, TH = cfg.tile_h;
    const int nq = TWE >> 2;                 // element quads per tile row
    const int rpp = blockDim.x / nq;         // rows per pass
    const int tid = threadIdx.x;
    const int qx = tid % nq, ty = tid / nq;

    const int64_t WoC = (int64_t)g.Wo * C;
    const int64_t e0 = (int64_t)bx * TWE;
    const int y0 = by * TH;
    const int nE = (int)min((int64_t)TWE, WoC - e0);
    const int nR = min(TH, g.Ho - y0);

    // Footprint of the tile in source pixels / rows (first taps are monotone).
    const int j_first = (int)(e0 / C), j_last = (int)((e0 + nE - 1) / C);
    const int px_lo = first_tap<KT>(j_first, g.W, g.Wo, g.coord);
    const int px_hi = first_tap<KT>(j_last, g.W, g.Wo, g.coord) + KT - 1;
    const int ry_lo = first_tap<KT>(y0, g.H, g.Ho, g.coord);
    const int ry_hi = first_tap<KT>(y0 + nR - 1, g.H, g.Ho, g.coord) + KT - 1;
    const int SWE = (px_hi - px_lo + 1) * C;
    const int SH = ry_hi - ry_lo + 1;
    if (SWE > cfg.swe_max || SH > cfg.sh_max) {   // uniform over the block
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }

    float* S = sm;                                   // [sh_max][swe_max]
    float* Hb = S + cfg.sh_max * cfg.swe_max;        // [sh_max][TWE]
    float* RW = Hb + cfg.sh_max * TWE;               // [TH][KT]
    int* RB = reinterpret_cast<int*>(RW + TH * KT);  // [TH]

    // 1. Row taps.
    for (int i = tid; i < nR; i += blockDim.x) {
        float w[KT];
        const int f = taps<KT>(y0 + i, g.H, g.Ho, g.coord, g.a, w);
        RB[i] = f - ry_lo;
        #pragma unroll
        for (int p = 0; p < KT; ++p) RW[i * KT + p] = w[p];
    }
    // Column taps of this thread's four elements (offsets into a staged row).
    int off[4];
    float wx[4][KT];
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int el = 4 * qx + k;
        if (el < nE) {
            const int64_t e = e0 + el;
            const int j = (int)(e / C), c = (int)(e - (int64_t)j * C);
            const int f = taps<KT>(j, g.W, g.Wo, g.coord, g.a, wx[k]);
            off[k] = (f - px_lo) * C + c;
        } else {
            off[k] = 0;
            #pragma unroll
            for (int q = 0; q < KT; ++q) wx[k][q] = 0.0f;
        }
    }

    // 2. Stage the clamped source footprint as FP32.
    {
        const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
        for (int r = warp; r < SH; r += nwarps) {
            const int row = clampi(ry_lo + r, g.H);
            const T* srow = s + (int64_t)row * g.src_pitch;
            float* Sr = S + r * cfg.swe_max;
            for (int ce = lane; ce < SWE; ce += 32) {
                const int px = ce / C, c = ce - px * C;
                const int sx = clampi(px_lo + px, g.W);
                Sr[ce] = Store<T>::load(srow + (int64_t)sx * C + c);
            }
        }
    }
    __syncthreads();

    // 3. Horizontal pass.
    const bool active = 4 * qx < nE;
    if (active && ty < rpp) {
        for (int r = ty; r < SH; r += rpp) {
            const float* Sr = S + r * cfg.swe_max;
            float h[4];
            #pragma unroll
            for (int k = 0; k < 4; ++k) {
                float acc = 0.0f;
                #pragma unroll
                for (int q = 0; q < KT; ++q) acc = fmaf(wx[k][q], Sr[off[k] + q * C], acc);
                h[k] = acc;
            }
            *reinterpret_cast<float4*>(Hb + r * TWE + 4 * qx) = make_float4(h[0], h[1], h[2], h[3]);
        }
    }
    __syncthreads();

    // 4. Vertical pass and store.
    if (active && ty < rpp) {
        const int cnt = min(4, nE - 4 * qx);
        for (int i = ty; i < nR; i += rpp) {
            const int b = RB[i];
            float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            #pragma unroll
            for (int p = 0; p < KT; ++p) {
                const float wy = RW[i * KT + p];
                const float4 hv = *reinterpret_cast<const float4*>(Hb + (b + p) * TWE + 4 * qx);
                v[0] = fmaf(wy, hv.x, v[0]);
                v[1] = fmaf(wy, hv.y, v[1]);
                v[2] = fmaf(wy, hv.z, v[2]);
                v[3] = fmaf(wy, hv.w, v[3]);
            }
            store4<T>(d + (int64_t)(y0 + i) * g.dst_pitch + e0 + 4 * qx, v, cnt);
        }
    }
}

}  // namespace rs
