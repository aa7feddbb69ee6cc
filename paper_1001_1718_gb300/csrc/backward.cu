// Backward (adjoint) of the forward resampling, in gather form.
//
// The forward is a separable linear map: per plane Y = Ay X Ax^T, where row
// j of an axis matrix holds output j's tap weights at the clamped source
// indices. The gradient is dX = Ay^T dY Ax. Row i of A^T is sparse and
// contiguous: since the first tap index of output j never decreases with j,
// the outputs whose taps land on input i form one range [jlo(i), jhi(i)];
// border inputs also receive the clamped taps, which only widens their range.
//
// 1. k_adjoint_tables builds, for both axes in one launch, jlo(i), the range
//    length and the summed weights w(i, j) = sum over taps q of output j with
//    clamp(first(j) + q) == i, into the caller's workspace.
// 2. Default: two memory-bound passes per group of planes through an FP32
//    intermediate T in the workspace: k_adj_x applies the x-axis transpose to
//    every dY row (T = dY Ax, Ho x W), k_adj_y the y-axis transpose
//    (dX = Ay^T T). Both are coalesced along rows; each thread keeps its
//    column's (or row's) transposed weights in registers and walks several
//    rows. Alternatively (RS_IMPL_TILED) k_adjoint computes a tile of dX in
//    one pass: it stages the dY footprint of the tile in shared memory,
//    applies the x-axis transpose to every staged row, then the y-axis
//    transpose. Every dX element is one fixed-order sum, so the result is
//    deterministic (no atomics).
#include <algorithm>
#include <climits>
#include <vector>

#include "capi_internal.h"
#include "rs_common.cuh"

namespace rs {

// Exact first tap index on the host (same integer arithmetic as the device).
static int64_t host_floor_div(int64_t num, int64_t den)
{
    int64_t q = num / den;
    if ((num % den != 0) && (num < 0)) q -= 1;
    return q;
}

static int host_first_tap(int j, int n, int m, int method, int coord)
{
    if (coord == COORD_ALIGN_CORNERS) {   // x = j (n - 1) / (m - 1); 0 for one output
        const int64_t num = m > 1 ? (int64_t)j * (n - 1) : 0, den = m > 1 ? m - 1 : 1;
        if (method == M_NEAREST) return (int)host_floor_div(2 * num + den, 2 * den);
        const int64_t i0 = host_floor_div(num, den);
        return (int)(method == M_BICUBIC ? i0 - 1 : i0);
    }
    if (method == M_NEAREST) {
        if (coord == COORD_ASYMMETRIC) return (int)host_floor_div((int64_t)j * n, m);
        return (int)host_floor_div((int64_t)(2 * j + 1) * n, 2 * (int64_t)m);
    }
    int64_t i0 = coord == COORD_ASYMMETRIC ? host_floor_div((int64_t)j * n, m)
                                           : host_floor_div((int64_t)(2 * j + 1) * n - m, 2 * (int64_t)m);
    return (int)(method == M_BICUBIC ? i0 - 1 : i0);
}

// Ranges [lo[i], hi[i]] of outputs touching input i (hi < lo when none).
struct AxisRanges {
    std::vector<int> lo, hi;
    int kmax = 0;
};

static AxisRanges host_ranges(int n, int m, int method, int coord)
{
    const int KT = method_taps(method);
    std::vector<int> first(m);
    for (int j = 0; j < m; ++j) first[j] = host_first_tap(j, n, m, method, coord);
    AxisRanges R;
    R.lo.resize(n);
    R.hi.resize(n);
    for (int i = 0; i < n; ++i) {
        // contributors: first(j) in [lo_i, hi_i] with the border widening
        const int64_t lo_i = (i == 0) ? INT32_MIN : (int64_t)i - KT + 1;
        const int64_t hi_i = (i == n - 1) ? INT32_MAX : (int64_t)i;
        const int jl = (int)(std::lower_bound(first.begin(), first.end(), lo_i) - first.begin());
        const int jh = (int)(std::upper_bound(first.begin(), first.end(), hi_i) - first.begin()) - 1;
        R.lo[i] = jl;
        R.hi[i] = jh;
        R.kmax = std::max(R.kmax, jh - jl + 1);
    }
    return R;
}

// Antialias taps (method aa): outputs j with lo(j) <= i < hi(j).
static AxisRanges host_ranges_aa(int n, int m, int aa)
{
    std::vector<int> lo(m), hi(m);
    for (int j = 0; j < m; ++j) aa_range(j, n, m, aa, lo[j], hi[j]);
    AxisRanges R;
    R.lo.resize(n);
    R.hi.resize(n);
    for (int i = 0; i < n; ++i) {
        const int jl = (int)(std::upper_bound(hi.begin(), hi.end(), i) - hi.begin());
        const int jh = (int)(std::upper_bound(lo.begin(), lo.end(), i) - lo.begin()) - 1;
        R.lo[i] = jl;
        R.hi[i] = jh;
        R.kmax = std::max(R.kmax, jh - jl + 1);
    }
    return R;
}

__device__ __forceinline__ int first_tap_rt(int j, int n, int m, int method, int coord)
{
    if (method == M_NEAREST) return first_tap<1>(j, n, m, coord);
    if (method == M_BILINEAR) return first_tap<2>(j, n, m, coord);
    return first_tap<4>(j, n, m, coord);
}

__device__ __forceinline__ int taps_rt(int j, int n, int m, int method, int coord, float a, float* w)
{
    if (method == M_NEAREST) return taps<1>(j, n, m, coord, a, w);
    if (method == M_BILINEAR) return taps<2>(j, n, m, coord, a, w);
    return taps<4>(j, n, m, coord, a, w);
}

// One thread per input index i of an axis (n inputs, m outputs).
// One thread per (input index i, range slot k) of both axes in one launch:
// entries [0, ny * yK) are the y axis, the rest the x axis. Each thread finds
// i's output range [jlo, jhi] by binary search over the (non-decreasing)
// first taps and writes slot k's summed weight; slot 0 also writes jlo and
// the range length.
struct TableAxis {
    int n, m;          // inputs, outputs along the axis
    int K;             // slots per input
    int* lo;
    int* cnt;
    float* w;
};

// aa != 0: the antialias taps of method aa (RS_FLAG_ANTIALIAS); their
// ranges [lo(j), hi(j)) never decrease with j and lie inside the image, so
// input i's outputs are those with hi(j) > i and lo(j) <= i.
__global__ void k_adjoint_tables(TableAxis ya, TableAxis xa, int method, int coord, float a, int aa,
                                 unsigned int* fault)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ny = (int64_t)ya.n * ya.K;
    if (t >= ny + (int64_t)xa.n * xa.K) return;
    const TableAxis& ax = t < ny ? ya : xa;
    const int64_t u = t < ny ? t : t - ny;
    const int i = (int)(u / ax.K), k = (int)(u - (int64_t)i * ax.K);
    const int n = ax.n, m = ax.m;
    if (aa) {
        int l = 0, h = m, lo, hi;
        while (l < h) {   // first j with hi(j) > i
            const int mid = (l + h) >> 1;
            aa_range(mid, n, m, aa, lo, hi);
            if (hi > i) h = mid; else l = mid + 1;
        }
        const int jl = l;
        h = m;
        while (l < h) {   // first j with lo(j) > i
            const int mid = (l + h) >> 1;
            aa_range(mid, n, m, aa, lo, hi);
            if (lo > i) h = mid; else l = mid + 1;
        }
        int cnt = max(0, l - jl);
        if (cnt > ax.K) {
            if (k == 0) report_fault(fault, FAULT_BWD_TAPS);
            cnt = ax.K;
        }
        if (k == 0) {
            ax.lo[i] = jl;
            ax.cnt[i] = cnt;
        }
        ax.w[(int64_t)i * ax.K + k] = k < cnt ? aa_weight(jl + k, i, n, m, aa, a) : 0.0f;
        return;
    }
    const int KT = method == M_NEAREST ? 1 : method == M_BILINEAR ? 2 : 4;
    // jlo = first j with first(j) >= i - KT + 1 (0 for i == 0)
    int jl = 0;
    if (i > 0) {
        int l = 0, h = m;
        while (l < h) {
            const int mid = (l + h) >> 1;
            if (first_tap_rt(mid, n, m, method, coord) >= i - KT + 1) h = mid; else l = mid + 1;
        }
        jl = l;
    }
    // jhi = last j with first(j) <= i (m - 1 for i == n - 1)
    int jh = m - 1;
    if (i < n - 1) {
        int l = jl, h = m;
        while (l < h) {
            const int mid = (l + h) >> 1;
            if (first_tap_rt(mid, n, m, method, coord) > i) h = mid; else l = mid + 1;
        }
        jh = l - 1;
    }
    int cnt = max(0, jh - jl + 1);
    if (cnt > ax.K) {
        if (k == 0) report_fault(fault, FAULT_BWD_TAPS);
        cnt = ax.K;
    }
    if (k == 0) {
        ax.lo[i] = jl;
        ax.cnt[i] = cnt;
    }
    float acc = 0.0f;
    if (k < cnt) {
        float w[4];
        const int f = taps_rt(jl + k, n, m, method, coord, a, w);
        for (int q = 0; q < KT; ++q)
            if (clampi(f + q, n) == i) acc += w[q];
    }
    ax.w[(int64_t)i * ax.K + k] = acc;
}

struct AdjTables {
    const int *ylo, *ycnt, *xlo, *xcnt;
    const float *yw, *xw;
    int yK, xK;
};

struct AdjCfg {
    int tile_w, tile_h, ty;   // dX elements per tile row (= blockDim.x), dX rows per tile, blockDim.y
    int fh_max, fwe_max;      // staged dY footprint bound
    size_t smem;
};

// g describes the FORWARD problem: H x W inputs (dX), Ho x Wo outputs (dY).
template <int KX, int C>
__global__ void __launch_bounds__(256)
k_adjoint(const Geom g, const float* __restrict__ dY, float* __restrict__ dX, const AdjTables tb,
          const AdjCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int tx = threadIdx.x, ty = threadIdx.y, TY = blockDim.y;
    const int tid = ty * blockDim.x + tx, nthreads = blockDim.x * TY;
    const int TWE = cfg.tile_w, TH = cfg.tile_h;
    const int plane = blockIdx.z;
    const float* s = dY + g.dp.offset(plane);   // dY has the output layout
    float* d = dX + g.sp.offset(plane);

    const int64_t WC = (int64_t)g.W * C;
    const int64_t e0 = (int64_t)blockIdx.x * TWE;
    const int i0 = blockIdx.y * TH;
    const int nE = (int)min((int64_t)TWE, WC - e0);
    const int nR = min(TH, g.H - i0);
    const int x_first = (int)(e0 / C), x_last = (int)((e0 + nE - 1) / C);

    // Footprint in dY (ranges are monotone; empty ranges have cnt 0).
    int r_lo = tb.ylo[i0], r_hi = tb.ylo[i0 + nR - 1] + tb.ycnt[i0 + nR - 1] - 1;
    int c_lo = tb.xlo[x_first], c_hi = tb.xlo[x_last] + tb.xcnt[x_last] - 1;
    r_hi = max(r_hi, r_lo);     // keep at least one staged row / column
    c_hi = max(c_hi, c_lo);
    r_lo = min(r_lo, g.Ho - 1);
    r_hi = min(r_hi, g.Ho - 1);
    c_lo = min(c_lo, g.Wo - 1);
    c_hi = min(c_hi, g.Wo - 1);
    const int FH = r_hi - r_lo + 1, FWE = (c_hi - c_lo + 1) * C;
    if (FH > cfg.fh_max || FWE > cfg.fwe_max) {
        if (tid == 0) report_fault(fault, FAULT_BWD_SPAN);
        return;
    }
    float* S = sm;                                  // [fh_max][fwe_max]
    float* Hb = S + cfg.fh_max * cfg.fwe_max;       // [fh_max][TWE]
    float* RW = Hb + cfg.fh_max * TWE;              // [TH][yK]
    int* RL = reinterpret_cast<int*>(RW + TH * tb.yK);   // [TH] first staged row
    int* RC = RL + TH;                                   // [TH] count

    for (int i = tid; i < nR; i += nthreads) {
        RL[i] = tb.ylo[i0 + i] - r_lo;
        RC[i] = tb.ycnt[i0 + i];
        for (int k = 0; k < tb.yK; ++k) RW[i * tb.yK + k] = tb.yw[(int64_t)(i0 + i) * tb.yK + k];
    }
    // this thread's dX element: its x-axis range and weights
    const bool active = tx < nE;
    int xoff = 0, xcnt = 0;
    float wx[KX];
    #pragma unroll
    for (int k = 0; k < KX; ++k) wx[k] = 0.0f;
    if (active) {
        const int64_t e = e0 + tx;
        const int x = (int)(e / C), c = (int)(e - (int64_t)x * C);
        xoff = (tb.xlo[x] - c_lo) * C + c;
        xcnt = min(tb.xcnt[x], KX);
        #pragma unroll
        for (int k = 0; k < KX; ++k)
            if (k < xcnt) wx[k] = tb.xw[(int64_t)x * tb.xK + k];
    }
    // stage the dY footprint
    for (int r = tid / 32; r < FH; r += nthreads / 32) {
        const float* srow = s + (int64_t)(r_lo + r) * g.dst_pitch + (int64_t)c_lo * C;
        float* Sr = S + r * cfg.fwe_max;
        for (int ce = tid % 32; ce < FWE; ce += 32) Sr[ce] = __ldg(srow + ce);
    }
    __syncthreads();
    // x-axis transpose of every staged row
    if (active) {
        for (int r = ty; r < FH; r += TY) {
            const float* Sr = S + r * cfg.fwe_max + xoff;
            float acc = 0.0f;
            #pragma unroll
            for (int k = 0; k < KX; ++k)
                if (k < xcnt) acc = fmaf(wx[k], Sr[k * C], acc);
            Hb[r * TWE + tx] = acc;
        }
    }
    __syncthreads();
    // y-axis transpose and store
    if (active) {
        for (int i = ty; i < nR; i += TY) {
            const int b = RL[i], cnt = RC[i];
            const float* w = RW + i * tb.yK;
            float acc = 0.0f;
            for (int k = 0; k < cnt; ++k) acc = fmaf(w[k], Hb[(b + k) * TWE + tx], acc);
            d[(int64_t)(i0 + i) * g.src_pitch + e0 + tx] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Two-pass adjoint.

static constexpr int kAdjThreads = 256;

// T[p][j][e] = sum_k wx[x][k] dY[p][j][(xlo(x) + k) C + c] for the dY rows
// j of this block (e = x C + c). T has rows of W C elements. RU dY rows are
// gathered per iteration (independent loads in flight); row offsets within
// a plane are 32-bit (the host bounds Ho x pitch below 2^31).
template <int KXM, int RU>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_x(const Geom g, const float* __restrict__ dY, float* __restrict__ T, const AdjTables tb, int plane0,
        int rows_per_thread)
{
    const int WC = g.W * g.C;
    const int e = blockIdx.x * kAdjThreads + threadIdx.x;
    if (e >= WC) return;
    const int pl = blockIdx.z;
    const int x = e / g.C, c = e - x * g.C;
    const int lo = __ldg(tb.xlo + x);
    const int cnt = min(__ldg(tb.xcnt + x), KXM);
    float w[KXM];
    #pragma unroll
    for (int k = 0; k < KXM; ++k) w[k] = k < cnt ? __ldg(tb.xw + (int64_t)x * tb.xK + k) : 0.0f;
    const float* src = dY + g.dp.offset(plane0 + pl) + lo * g.C + c;
    float* dst = T + (int64_t)pl * g.Ho * WC + e;
    const int pitch = (int)g.dst_pitch;
    const int j0 = blockIdx.y * rows_per_thread, j1 = min(g.Ho, j0 + rows_per_thread);
    int j = j0;
    for (; j + RU <= j1; j += RU) {
        float acc[RU];
        #pragma unroll
        for (int r = 0; r < RU; ++r) acc[r] = 0.0f;
        #pragma unroll
        for (int k = 0; k < KXM; ++k) {
            if (k < cnt) {
                float v[RU];
                #pragma unroll
                for (int r = 0; r < RU; ++r) v[r] = __ldg(src + (j + r) * pitch + k * g.C);
                #pragma unroll
                for (int r = 0; r < RU; ++r) acc[r] = fmaf(w[k], v[r], acc[r]);
            }
        }
        #pragma unroll
        for (int r = 0; r < RU; ++r) dst[(j + r) * WC] = acc[r];
    }
    for (; j < j1; ++j) {
        const float* row = src + j * pitch;
        float acc = 0.0f;
        #pragma unroll
        for (int k = 0; k < KXM; ++k)
            if (k < cnt) acc = fmaf(w[k], __ldg(row + k * g.C), acc);
        dst[j * WC] = acc;
    }
}

// dX[p][i][e..e+V-1] = sum_a wy[i][a] T[p][ylo(i) + a][e..e+V-1] for the dX
// rows i of this block; V = 4 (16-byte loads and stores) when rows allow.
template <int KYM, int V>
__global__ void __launch_bounds__(kAdjThreads)
k_adj_y(const Geom g, const float* __restrict__ T, float* __restrict__ dX, const AdjTables tb, int plane0,
        int rows_per_thread)
{
    const int WC = g.W * g.C;
    const int e = (blockIdx.x * kAdjThreads + threadIdx.x) * V;
    if (e >= WC) return;
    const int pl = blockIdx.z;
    const float* src = T + (int64_t)pl * g.Ho * WC + e;
    float* dst = dX + g.sp.offset(plane0 + pl) + e;
    const int pitch = (int)g.src_pitch;
    const int i0 = blockIdx.y * rows_per_thread, i1 = min(g.H, i0 + rows_per_thread);
    for (int i = i0; i < i1; ++i) {
        const int lo = __ldg(tb.ylo + i), cnt = min(__ldg(tb.ycnt + i), KYM);
        const float* wr = tb.yw + (int64_t)i * tb.yK;
        float acc[V];
        #pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        #pragma unroll
        for (int a = 0; a < KYM; ++a) {
            if (a < cnt) {
                const float wa = __ldg(wr + a);
                const float* row = src + (lo + a) * WC;
                if constexpr (V == 4) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(row));
                    acc[0] = fmaf(wa, t.x, acc[0]);
                    acc[1] = fmaf(wa, t.y, acc[1]);
                    acc[2] = fmaf(wa, t.z, acc[2]);
                    acc[3] = fmaf(wa, t.w, acc[3]);
                } else {
                    acc[0] = fmaf(wa, __ldg(row), acc[0]);
                }
            }
        }
        if constexpr (V == 4) *reinterpret_cast<float4*>(dst + i * pitch) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        else dst[i * pitch] = acc[0];
    }
}

// ---------------------------------------------------------------------------
// Fused register-window adjoint (FP32, dY rows of whole 16-byte units).
//
// The transpose of the forward's register window. A block of NT threads
// owns a strip of 2 NT dX elements and a band of dX rows; thread t owns
// elements t and t + NT. It walks the rows of T = dY Ax that the band's y taps reach
// ("positions"): each dY row, staged in shared memory, is x-adjointed at
// the thread's two columns into a register window of the last KY such
// rows, and every dX row whose first y tap is the window's first row is
// blended from registers and stored. dY rows are copied with 16-byte
// cp.async in chunks of R rows into a three-slot ring two chunks ahead and
// read in place. The sums run in the two-pass order (x taps, then y taps,
// each ascending), so the results equal the two-pass kernels'.
struct AdjWinCfg {
    int band_h, band_cap, pos_cap, chunk, swe_max;
    int nt;          // threads per block (strips of 2 nt dX elements)
    int tap_method;  // computed taps (TAPS_AA, TAPS_POINT): M_BILINEAR / M_BICUBIC
    float tap_a;     // Keys parameter of the bicubic kernel
    size_t smem;
};

// Threads per block: 256 (strips of 512 dX elements), or 128 (strips of
// 256) for the computed-tap modes where that pads narrow rows less.
static constexpr int kAwThreads = 256;

// Where the taps come from. TAPS_TABLE: the transposed tables of the
// adjoint. TAPS_AA / TAPS_POINT: the same pass as a forward resampling, the
// "dY" rows being the source image and the "dX" rows the output, with the
// taps computed from the definition: antialias taps (the stretched kernel),
// or the point-sampled taps of Eqs. 1-5. Point taps keep the rows' clamped
// virtual indices (the staging clamps rows) and, along x, merge the weights
// of taps that clamp onto the same column, so that every output reads KX
// consecutive staged columns from max(first tap, 0).
enum { TAPS_TABLE = 0, TAPS_AA = 1, TAPS_POINT = 2 };

template <int C, int KX, int KY, int TM, int NT = kAwThreads>
__global__ void __launch_bounds__(NT, 512 / NT)
k_adj_window(const Geom g, const float* __restrict__ dY, float* __restrict__ dX, const AdjTables tb,
             const AdjWinCfg cfg, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;
    const float* s = dY + g.dp.offset(plane);   // Ho rows of Wo C, pitch dst_pitch
    float* d = dX + g.sp.offset(plane);         // H rows of W C, pitch src_pitch
    const int WC = g.W * C, WoC = g.Wo * C;
    const int e0 = blockIdx.x * (2 * NT);
    const int nE = min((2 * NT), WC - e0);
    const int yb = blockIdx.y * cfg.band_h;
    const int nrows = min(cfg.band_h, g.H - yb);

    // dY columns under the strip: [a0, c_hi), a0 on a 16-byte boundary; the
    // columns past the row (x taps beyond a range, zero weights) read zeros.
    const int x_first = e0 / C, x_last = (e0 + nE - 1) / C;
    auto xlo_of = [&](int x) {
        if constexpr (TM == TAPS_AA) {
            int lo, hi;
            aa_range(x, g.Wo, g.W, cfg.tap_method, lo, hi);
            return lo;
        } else if constexpr (TM == TAPS_POINT) {
            return max(first_tap<KX>(x, g.Wo, g.W, g.coord), 0);
        } else {
            return __ldg(tb.xlo + x);
        }
    };
    const int a0 = (xlo_of(x_first) * C) & ~3;
    const int c_hi = (xlo_of(x_last) + KX) * C;
    const int in_hi = min(c_hi, WoC);
    const int units = (in_hi - a0 + 3) / 4;
    const int R = cfg.chunk;
    if (c_hi - a0 > cfg.swe_max || nrows > cfg.band_cap || R < KY || R % KY) {   // uniform
        if (tid == 0) report_fault(fault, FAULT_BWD_SPAN);
        return;
    }
    float* RING = sm;                                            // [3][R][swe_max]
    float* RW = RING + 3 * R * cfg.swe_max;                      // [band_cap][KY]
    int* RF = reinterpret_cast<int*>(RW + cfg.band_cap * KY);    // [band_cap] first y taps
    int* NC = RF + cfg.band_cap;                                 // [pos_cap] rows per position
    if (c_hi > WoC) {
        const int z0 = WoC - a0, zn = c_hi - WoC;
        for (int u = tid; u < 3 * R * zn; u += NT) {
            const int row = u / zn;
            RING[row * cfg.swe_max + z0 + (u - row * zn)] = 0.0f;
        }
    }
    for (int i = tid; i < nrows; i += NT) {
        const int r = yb + i;
        if constexpr (TM == TAPS_AA) {
            float w[KY];
            aa_taps<KY>(r, g.Ho, g.H, cfg.tap_method, cfg.tap_a, RF[i], w, fault);
            #pragma unroll
            for (int p = 0; p < KY; ++p) RW[i * KY + p] = w[p];
        } else if constexpr (TM == TAPS_POINT) {
            float w[KY];
            RF[i] = taps<KY>(r, g.Ho, g.H, g.coord, cfg.tap_a, w);
            #pragma unroll
            for (int p = 0; p < KY; ++p) RW[i * KY + p] = w[p];
        } else {
            RF[i] = __ldg(tb.ylo + r);
            const int cnt = __ldg(tb.ycnt + r);
            #pragma unroll
            for (int p = 0; p < KY; ++p) RW[i * KY + p] = p < cnt ? __ldg(tb.yw + (int64_t)r * tb.yK + p) : 0.0f;
        }
    }
    // x taps of this thread's two elements, paired for FP32x2
    int off[2];
    float2 wxp[KX];
    {
        float wx[2][KX];
        #pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int el = tid + NT * k;
            if (el < nE) {
                const int e = e0 + el, x = e / C, c = e - x * C;
                int lo;
                if constexpr (TM == TAPS_AA) {
                    aa_taps<KX>(x, g.Wo, g.W, cfg.tap_method, cfg.tap_a, lo, wx[k], fault);
                } else if constexpr (TM == TAPS_POINT) {
                    float wt[KX];
                    const int f = taps<KX>(x, g.Wo, g.W, g.coord, cfg.tap_a, wt);
                    lo = max(f, 0);
                    #pragma unroll
                    for (int q = 0; q < KX; ++q) wx[k][q] = 0.0f;
                    #pragma unroll
                    for (int q = 0; q < KX; ++q) {   // tap q lands on column lo + dq
                        const int dq = clampi(f + q, g.Wo) - lo;
                        #pragma unroll
                        for (int t = 0; t < KX; ++t) wx[k][t] += dq == t ? wt[q] : 0.0f;
                    }
                } else {
                    lo = __ldg(tb.xlo + x);
                    const int cnt = __ldg(tb.xcnt + x);
                    #pragma unroll
                    for (int q = 0; q < KX; ++q) wx[k][q] = q < cnt ? __ldg(tb.xw + (int64_t)x * tb.xK + q) : 0.0f;
                }
                off[k] = lo * C + c - a0;
            } else {
                off[k] = 0;
                #pragma unroll
                for (int q = 0; q < KX; ++q) wx[k][q] = 0.0f;
            }
        }
        #pragma unroll
        for (int q = 0; q < KX; ++q) wxp[q] = make_float2(wx[0][q], wx[1][q]);
    }
    for (int p = tid; p < cfg.pos_cap; p += NT) NC[p] = 0;
    __syncthreads();
    const int b_first = RF[0], b_last = RF[nrows - 1];
    if (b_last - b_first + 1 > cfg.pos_cap) {   // uniform; the host bounds the positions
        if (tid == 0) report_fault(fault, FAULT_BWD_SPAN);
        return;
    }
    for (int i0 = tid; i0 < nrows; i0 += NT) {
        if (i0 == 0 || RF[i0] != RF[i0 - 1]) {
            int len = 1;
            while (i0 + len < nrows && RF[i0 + len] == RF[i0]) ++len;
            NC[RF[i0] - b_first] = len;
        }
    }
    // dY rows b_first .. b_last + KY - 1 (past the last row: the last row,
    // under zero weights), in chunks of R.
    const int r_first = b_first, r_end = b_last + KY;
    auto chunk_rows = [&](int c) { return max(0, min(R, r_end - (r_first + c * R))); };
    const uint32_t umul = units > 1 ? 0xFFFFFFFFu / (uint32_t)units + 1u : 0u;
    auto issue = [&](int c) {
        const int r0 = r_first + c * R, nn = chunk_rows(c);
        float* slot = RING + (c % 3) * R * cfg.swe_max;
        for (int u = tid; u < nn * units; u += NT) {
            const int k = units > 1 ? (int)__umulhi((uint32_t)u, umul) : u;
            const int w = u - k * units;
            const float* src = s + (int64_t)clampi(r0 + k, g.Ho) * g.dst_pitch + a0 + 4 * w;
            const unsigned sdst = (unsigned)__cvta_generic_to_shared(slot + k * cfg.swe_max + 4 * w);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    issue(1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();   // chunk 0 and the position table visible
    issue(2);

    // One channel: a thread's KX taps are consecutive floats, read as KX / 2
    // + 1 8-byte pairs from the even float at or below the first tap (the
    // odd-offset threads take the taps one float on), so neighbouring
    // threads' taps, two floats apart at a x2 upscale, cost no bank conflicts.
    // The last pair may reach one float past the staged row (still inside
    // the block's shared memory) and is then not used.
    constexpr bool pairs = C == 1 && KX % 2 == 0;
    int pb[2];
    bool podd[2];
    #pragma unroll
    for (int k = 0; k < 2; ++k) {
        pb[k] = off[k] & ~1;
        podd[k] = off[k] & 1;
    }
    auto hrow = [&](const float* Sr, float2& h) {
        h = make_float2(0.0f, 0.0f);
        if constexpr (pairs) {
            float e[2][KX + 2];
            #pragma unroll
            for (int k = 0; k < 2; ++k)
                #pragma unroll
                for (int t = 0; t < KX / 2 + 1; ++t) {
                    const float2 v = reinterpret_cast<const float2*>(Sr + pb[k])[t];
                    e[k][2 * t] = v.x;
                    e[k][2 * t + 1] = v.y;
                }
            #pragma unroll
            for (int q = 0; q < KX; ++q)
                h = __ffma2_rn(wxp[q], make_float2(podd[0] ? e[0][q + 1] : e[0][q], podd[1] ? e[1][q + 1] : e[1][q]), h);
        } else {
            #pragma unroll
            for (int q = 0; q < KX; ++q)
                h = __ffma2_rn(wxp[q], make_float2(Sr[off[0] + q * C], Sr[off[1] + q * C]), h);
        }
    };
    float2 h[KY];
    #pragma unroll
    for (int p = 0; p < KY - 1; ++p) hrow(RING + p * cfg.swe_max, h[p]);
    int r = b_first + KY - 1, cidx = 0, chunk_lo = r_first;
    int nn = chunk_rows(0);
    int i = 0, b = b_first;
    const int nact = (tid < nE) + (tid + NT < nE);
    float* const dband = d + (int64_t)yb * g.src_pitch + e0 + tid;
    const int pitch32 = (int)g.src_pitch;
    auto blend_put = [&](int row, const int* slot) {
        // the row's KY weights in 16-byte (KY >= 4) or 8-byte loads: RW and
        // its rows of KY floats are 16-byte aligned
        float w[KY];
        if constexpr (KY % 4 == 0) {
            #pragma unroll
            for (int p = 0; p < KY; p += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(RW + row * KY + p);
                w[p] = w4.x; w[p + 1] = w4.y; w[p + 2] = w4.z; w[p + 3] = w4.w;
            }
        } else if constexpr (KY % 2 == 0) {
            #pragma unroll
            for (int p = 0; p < KY; p += 2) {
                const float2 w2 = *reinterpret_cast<const float2*>(RW + row * KY + p);
                w[p] = w2.x; w[p + 1] = w2.y;
            }
        } else {
            #pragma unroll
            for (int p = 0; p < KY; ++p) w[p] = RW[row * KY + p];
        }
        float2 v = make_float2(0.0f, 0.0f);
        #pragma unroll
        for (int p = 0; p < KY; ++p) v = __ffma2_rn(make_float2(w[p], w[p]), h[slot[p]], v);
        float* q = dband + row * pitch32;
        if (nact > 0) q[0] = v.x;
        if (nact > 1) q[NT] = v.y;
    };
    while (b <= b_last) {
        #pragma unroll
        for (int u = 0; u < KY; ++u) {
            if (b <= b_last) {
                // with R a multiple of KY a chunk is entered only at u == 1
                if (u == 1 % KY && r >= chunk_lo + nn) {
                    ++cidx;
                    chunk_lo = r_first + cidx * R;
                    nn = chunk_rows(cidx);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                    __syncthreads();   // chunk cidx visible; chunk cidx - 1 no longer read
                    issue(cidx + 2);
                }
                const int ns = (u + KY - 1) % KY;
                hrow(RING + ((cidx % 3) * R + (r - chunk_lo)) * cfg.swe_max, h[ns]);
                ++r;
                int slot[KY];
                #pragma unroll
                for (int p = 0; p < KY; ++p) slot[p] = (u + p) % KY;
                const int nb = NC[b - b_first];
                for (int k = 0; k < nb; ++k) blend_put(i + k, slot);
                i += nb;
                ++b;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct BwdPlan {
    AxisRanges ry, rx;
    int yK, xK;
    size_t ws_bytes;
    size_t off_ylo, off_ycnt, off_yw, off_xlo, off_xcnt, off_xw;
    size_t off_t;        // two-pass intermediate T (group_planes x Ho x W C floats)
    int group_planes;
};

static constexpr size_t kAdjTBudget = (size_t)256 << 20;  // bytes of T per plane group

static BwdPlan plan_tables(const Geom& g, int method, int aa)
{
    BwdPlan p;
    p.ry = aa ? host_ranges_aa(g.H, g.Ho, aa) : host_ranges(g.H, g.Ho, method, g.coord);
    p.rx = aa ? host_ranges_aa(g.W, g.Wo, aa) : host_ranges(g.W, g.Wo, method, g.coord);
    p.yK = std::max(1, p.ry.kmax);
    p.xK = std::max(1, p.rx.kmax);
    size_t o = 0;
    p.off_ylo = o; o = align256(o + sizeof(int) * g.H);
    p.off_ycnt = o; o = align256(o + sizeof(int) * g.H);
    p.off_yw = o; o = align256(o + sizeof(float) * (size_t)g.H * p.yK);
    p.off_xlo = o; o = align256(o + sizeof(int) * g.W);
    p.off_xcnt = o; o = align256(o + sizeof(int) * g.W);
    p.off_xw = o; o = align256(o + sizeof(float) * (size_t)g.W * p.xK);
    const size_t plane_t = sizeof(float) * (size_t)g.Ho * g.W * g.C;
    p.group_planes = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.planes, kAdjTBudget / plane_t));
    p.off_t = o; o = align256(o + plane_t * p.group_planes);
    p.ws_bytes = o;
    return p;
}

// Largest staged footprint over all tiles of `tile` destination indices
// (rows: tile = TH; columns: element tiles of TWE over C channels).
static int footprint_bound(const AxisRanges& R, int n, int tile, int C, int m)
{
    int best = 1;
    const int64_t total = (int64_t)n * C;
    for (int64_t e0 = 0; e0 < total; e0 += tile) {
        const int first = (int)(e0 / C);
        const int last = (int)(std::min(total, e0 + tile) - 1) / C;
        int lo = R.lo[first], hi = R.hi[last];
        hi = std::max(hi, lo);
        lo = std::min(lo, m - 1);
        hi = std::min(hi, m - 1);
        best = std::max(best, hi - lo + 1);
    }
    return best;
}

static bool adj_config(const Geom& g, const BwdPlan& p, int TH, AdjCfg& cfg)
{
    cfg.tile_w = 128;
    cfg.ty = 2;
    cfg.tile_h = TH;
    cfg.fh_max = footprint_bound(p.ry, g.H, TH, 1, g.Ho);
    cfg.fwe_max = (footprint_bound(p.rx, g.W, cfg.tile_w, g.C, g.Wo) * g.C + 3) & ~3;
    cfg.smem = sizeof(float) * ((size_t)cfg.fh_max * cfg.fwe_max + (size_t)cfg.fh_max * cfg.tile_w +
                                (size_t)TH * p.yK) + sizeof(int) * 2 * (size_t)TH;
    return cfg.smem <= max_smem_per_block();
}

static int adj_taps_class(int k) { return k <= 2 ? 2 : k <= 4 ? 4 : 8; }

// The fused window adjoint applies with at most 8 transposed taps per axis,
// dY rows of whole 16-byte units and a footprint that fits shared memory.
static bool adj_window_config(const Geom& g, const BwdPlan& p, const void* dY, AdjWinCfg& c, bool narrow = false)
{
    if (p.xK > 8 || p.yK > 8) return false;
    const int KX = adj_taps_class(p.xK), KY = adj_taps_class(p.yK);
    if (reinterpret_cast<uintptr_t>(dY) % 16 || g.dst_pitch % 4 || ((int64_t)g.Wo * g.C) % 4) return false;
    if (g.planes > 1 && (g.dp.n_stride % 4 || g.dp.c_stride % 4)) return false;
    c.chunk = std::max(4, KY);
    const int WC = g.W * g.C;
    // 128-thread blocks where strips of 256 pad the rows less than strips of 512
    c.nt = narrow && (WC + 255) / 256 * 256 < (WC + 511) / 512 * 512 ? 128 : kAwThreads;
    const int elems = 2 * c.nt;
    int swe = 4;
    for (int e0 = 0; e0 < WC; e0 += elems) {
        const int nE = std::min(elems, WC - e0);
        const int xf = e0 / g.C, xl = (e0 + nE - 1) / g.C;
        const int a0 = (p.rx.lo[xf] * g.C) & ~3;
        swe = std::max(swe, (p.rx.lo[xl] + KX) * g.C - a0);
    }
    c.swe_max = (swe + 3) & ~3;
    c.band_cap = std::min(256, g.H);
    int pos = 1;
    for (int i = 0; i < g.H; ++i) {
        const int last = std::min(g.H - 1, i + c.band_cap - 1);
        pos = std::max(pos, p.ry.lo[last] - p.ry.lo[i] + 1);
    }
    c.pos_cap = pos;
    if ((int64_t)c.band_cap * g.src_pitch >= (int64_t)INT32_MAX) return false;   // 32-bit row offsets
    c.smem = sizeof(float) * (3 * (size_t)c.chunk * c.swe_max + (size_t)c.band_cap * KY) +
             sizeof(int) * ((size_t)c.band_cap + (size_t)c.pos_cap);
    c.band_h = 0;
    return c.smem <= max_smem_per_block();
}

template <int C, int KX, int KY>
static void* adj_window_func(int tm, int nt)
{
    if (tm == TAPS_AA)
        return nt == 128 ? reinterpret_cast<void*>(&k_adj_window<C, KX, KY, TAPS_AA, 128>)
                         : reinterpret_cast<void*>(&k_adj_window<C, KX, KY, TAPS_AA>);
    return reinterpret_cast<void*>(&k_adj_window<C, KX, KY, TAPS_TABLE>);
}

template <int C, int KX>
static void* adj_window_fy(int KY, int tm, int nt)
{
    return KY == 2 ? adj_window_func<C, KX, 2>(tm, nt) : KY == 4 ? adj_window_func<C, KX, 4>(tm, nt)
                                                               : adj_window_func<C, KX, 8>(tm, nt);
}

template <int C>
static void* adj_window_fx(int KX, int KY, int tm, int nt)
{
    if (tm == TAPS_POINT) {   // the method's own taps on both axes: KX == KY in {2, 4}
        if (nt == 128)
            return KX == 2 ? reinterpret_cast<void*>(&k_adj_window<C, 2, 2, TAPS_POINT, 128>)
                           : reinterpret_cast<void*>(&k_adj_window<C, 4, 4, TAPS_POINT, 128>);
        return KX == 2 ? reinterpret_cast<void*>(&k_adj_window<C, 2, 2, TAPS_POINT>)
                       : reinterpret_cast<void*>(&k_adj_window<C, 4, 4, TAPS_POINT>);
    }
    return KX == 2 ? adj_window_fy<C, 2>(KY, tm, nt) : KX == 4 ? adj_window_fy<C, 4>(KY, tm, nt)
                                                               : adj_window_fy<C, 8>(KY, tm, nt);
}

static cudaError_t launch_adj_window(const Geom& g, const BwdPlan& p, const float* dY, float* dX, const AdjTables& tb,
                                     AdjWinCfg c, cudaStream_t st, int tm = TAPS_TABLE)
{
    const int KX = adj_taps_class(p.xK), KY = adj_taps_class(p.yK);
    if (tm == TAPS_POINT && (KX != KY || KX > 4)) return cudaErrorInvalidValue;
    if (c.nt != kAwThreads && (c.nt != 128 || tm == TAPS_TABLE)) return cudaErrorInvalidValue;
    void* func = g.C == 1 ? adj_window_fx<1>(KX, KY, tm, c.nt) : g.C == 2 ? adj_window_fx<2>(KX, KY, tm, c.nt)
               : g.C == 3 ? adj_window_fx<3>(KX, KY, tm, c.nt) : adj_window_fx<4>(KX, KY, tm, c.nt);
    int per_sm = 1;
    cudaError_t e = prepare_kernel(func, c.smem, c.nt, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t strips = ((int64_t)g.W * g.C + 2 * c.nt - 1) / (2 * c.nt);
    const int64_t resident = (int64_t)num_sms() * std::max(1, per_sm);
    const int64_t bands = std::max<int64_t>(1, 2 * resident / (strips * g.planes));   // no partial extra wave
    c.band_h = (int)std::min<int64_t>(c.band_cap, std::max<int64_t>(1, (g.H + bands - 1) / bands));
    dim3 grid((unsigned)strips, (unsigned)((g.H + c.band_h - 1) / c.band_h), (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<float**>(&dY), &dX, const_cast<AdjTables*>(&tb), &c, &fw};
    e = cudaLaunchKernel(func, grid, dim3(c.nt), args, c.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// A forward problem in the window pass's adjoint roles: "dY" (Ho x Wo
// there) is the source image, "dX" (H x W) the output.
static Geom forward_as_adjoint(const Geom& gf)
{
    Geom g = gf;
    g.H = gf.Ho; g.W = gf.Wo; g.Ho = gf.H; g.Wo = gf.W;
    g.sp = gf.dp; g.dp = gf.sp;
    g.src_pitch = gf.dst_pitch; g.dst_pitch = gf.src_pitch;
    return g;
}

// Host ranges of the antialias taps (the same integer bounds as the kernel).
static AxisRanges aa_ranges(int n, int m, int method)
{
    AxisRanges R;
    R.lo.resize(m);
    R.hi.resize(m);
    for (int j = 0; j < m; ++j) {
        int lo, hi;
        aa_range(j, n, m, method, lo, hi);
        R.lo[j] = lo;
        R.hi[j] = hi - 1;
        R.kmax = std::max(R.kmax, hi - lo);
    }
    return R;
}

// The antialiased window form's configuration: K = 4 or 8 taps per axis,
// chunks of 8 staged rows, else 4 (K = 4: large FP32 footprints), else 16.
static bool aa_window_setup(const Geom& gf, int method, int dtype, int& K, WinCfg& c)
{
    const int k = antialias_taps(gf, method);
    K = k <= 4 ? 4 : k <= 8 ? 8 : 0;
    if (!K) return false;
    for (int ch : {8, 4, 16}) {
        if (ch % K) continue;
        c = WinCfg{};
        c.chunk = ch;
        if (win_config_aa(gf, method, dtype, K, c)) return true;
    }
    return false;
}

rs_status resize_antialias(const Geom& gf, int method, int dtype, const void* src, void* dst, const rs_options& o,
                           cudaStream_t st)
{
    if (method != M_BILINEAR && method != M_BICUBIC) return RS_ERR_INVALID_ARG;
    if (o.impl != RS_IMPL_AUTO && o.impl != RS_IMPL_WINDOW && o.impl != RS_IMPL_REDUCE && o.impl != RS_IMPL_TILED &&
        o.impl != RS_IMPL_STREAM)
        return RS_ERR_INVALID_ARG;
    if (o.impl == RS_IMPL_TILED) {   // the many-tap tiled kernel on request
        AaWideCfg wc;
        if (!aa_wide_config(gf, method, wc)) return RS_ERR_UNSUPPORTED;
        return cuda_status(launch_aa_wide(gf, dtype, src, dst, wc, st));
    }
    if (o.impl == RS_IMPL_STREAM) {   // the vertical-first streaming kernel on request
        AaVsCfg vc;
        if (!aa_vs_config(gf, method, dtype, vc)) return RS_ERR_UNSUPPORTED;
        return cuda_status(launch_aa_vs(gf, dtype, src, dst, vc, st));
    }
    if (dtype == DT_F32 && o.impl != RS_IMPL_WINDOW) {
        // FP32: the fused pass in its transposed roles reads the rows in place
        const Geom g = forward_as_adjoint(gf);
        BwdPlan p;
        p.ry = aa_ranges(gf.H, gf.Ho, method);
        p.rx = aa_ranges(gf.W, gf.Wo, method);
        p.yK = std::max(1, p.ry.kmax);
        p.xK = std::max(1, p.rx.kmax);
        AdjWinCfg c;
        if (adj_window_config(g, p, src, c, true)) {
            c.tap_method = method;
            c.tap_a = o.cubic_a;
            return cuda_status(launch_adj_window(g, p, static_cast<const float*>(src), static_cast<float*>(dst),
                                                 AdjTables{}, c, st, TAPS_AA));
        }
        if (o.impl == RS_IMPL_REDUCE) return RS_ERR_UNSUPPORTED;
    }
    if (o.impl == RS_IMPL_REDUCE) return RS_ERR_UNSUPPORTED;
    // any dtype: the general window form with antialias taps (at most 8 per
    // axis), else the many-tap tiled kernel
    int K = 0;
    WinCfg c;
    if (aa_window_setup(gf, method, dtype, K, c)) {
        c.waves = o.waves;
        return cuda_status(launch_win_aa(gf, method, dtype, src, dst, K, c, st));
    }
    if (o.impl == RS_IMPL_WINDOW) return RS_ERR_UNSUPPORTED;
    AaVsCfg vc;
    if (aa_vs_config(gf, method, dtype, vc)) return cuda_status(launch_aa_vs(gf, dtype, src, dst, vc, st));
    AaWideCfg wc;
    if (!aa_wide_config(gf, method, wc)) return RS_ERR_UNSUPPORTED;
    return cuda_status(launch_aa_wide(gf, dtype, src, dst, wc, st));
}

rs_status resize_normalize_antialias(const Geom& g, int method, int out_dtype, const void* src, void* dst,
                                     const NormOut& no, const rs_options& o, cudaStream_t st)
{
    int K = 0;
    WinCfg c;
    if (aa_window_setup(g, method, DT_U8, K, c)) {
        c.waves = o.waves;
        return cuda_status(launch_win_aa_norm(g, method, out_dtype, src, dst, K, c, no, st));
    }
    if (o.impl == RS_IMPL_WINDOW) return RS_ERR_UNSUPPORTED;
    AaVsCfg vc;
    if (aa_vs_config(g, method, DT_U8, vc)) return cuda_status(launch_aa_vs_norm(g, out_dtype, src, dst, vc, no, st));
    AaWideCfg wc;
    if (!aa_wide_config(g, method, wc)) return RS_ERR_UNSUPPORTED;
    return cuda_status(launch_aa_wide_norm(g, out_dtype, src, dst, wc, no, st));
}

// Host ranges of the point taps in the window pass's forward roles: rows
// keep the unclamped first tap (the staging clamps rows), columns start at
// max(first tap, 0) (the kernel merges clamped taps), as in k_adj_window.
static AxisRanges point_ranges(int n, int m, int method, int coord, bool columns)
{
    const int K = method_taps(method);
    AxisRanges R;
    R.lo.resize(m);
    R.hi.resize(m);
    for (int j = 0; j < m; ++j) {
        const int f = host_first_tap(j, n, m, method, coord);
        R.lo[j] = columns ? std::max(f, 0) : f;
        R.hi[j] = R.lo[j] + K - 1;
    }
    R.kmax = K;
    return R;
}

// The forward resampling through the fused window pass in its transposed
// roles (RS_IMPL_REDUCE): FP32 bilinear / bicubic, source rows of whole
// 16-byte units. Returns false where it does not apply.
static bool reduce_setup(const Geom& gf, int method, int dtype, const void* src, Geom& g, BwdPlan& p, AdjWinCfg& c)
{
    if (dtype != DT_F32 || (method != M_BILINEAR && method != M_BICUBIC)) return false;
    g = forward_as_adjoint(gf);
    p.ry = point_ranges(gf.H, gf.Ho, method, gf.coord, false);
    p.rx = point_ranges(gf.W, gf.Wo, method, gf.coord, true);
    p.yK = p.xK = method_taps(method);
    if (!adj_window_config(g, p, src, c, true)) return false;
    c.tap_method = method;
    c.tap_a = gf.a;
    return true;
}

bool reduce_config(const Geom& gf, int method, int dtype, const void* src, size_t* smem)
{
    Geom g;
    BwdPlan p;
    AdjWinCfg c;
    if (!reduce_setup(gf, method, dtype, src, g, p, c)) return false;
    if (smem) *smem = c.smem;
    return true;
}

cudaError_t launch_reduce(const Geom& gf, int method, int dtype, const void* src, void* dst, cudaStream_t st)
{
    Geom g;
    BwdPlan p;
    AdjWinCfg c;
    if (!reduce_setup(gf, method, dtype, src, g, p, c)) return cudaErrorInvalidValue;
    return launch_adj_window(g, p, static_cast<const float*>(src), static_cast<float*>(dst), AdjTables{}, c, st,
                             TAPS_POINT);
}

template <int KX, int C>
static cudaError_t launch_adj(const Geom& g, const float* dY, float* dX, const AdjTables& tb, const AdjCfg& cfg,
                              cudaStream_t st)
{
    auto kern = k_adjoint<KX, C>;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), cfg.smem, cfg.tile_w * cfg.ty, nullptr);
    if (e != cudaSuccess) return e;
    dim3 block(cfg.tile_w, cfg.ty);
    dim3 grid((unsigned)(((int64_t)g.W * C + cfg.tile_w - 1) / cfg.tile_w), (unsigned)((g.H + cfg.tile_h - 1) / cfg.tile_h),
              (unsigned)g.planes);
    kern<<<grid, block, cfg.smem, st>>>(g, dY, dX, tb, cfg, fault_word());
    return cudaGetLastError();
}

template <int KX>
static cudaError_t launch_adj_c(const Geom& g, const float* dY, float* dX, const AdjTables& tb, const AdjCfg& cfg,
                                cudaStream_t st)
{
    switch (g.C) {
    case 1: return launch_adj<KX, 1>(g, dY, dX, tb, cfg, st);
    case 2: return launch_adj<KX, 2>(g, dY, dX, tb, cfg, st);
    case 3: return launch_adj<KX, 3>(g, dY, dX, tb, cfg, st);
    case 4: return launch_adj<KX, 4>(g, dY, dX, tb, cfg, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rs

using namespace rs;

static rs_status bwd_geom(const rs_layout* out, const rs_layout* in, rs_method method, const rs_options& o,
                          Geom& g)
{
    LayoutInfo li, lo;
    // The forward's input layout is `in` (dX) and its output layout is `out` (dY).
    return geom_from_layouts(in, out, RS_F32, method, o, g, li, lo);
}

// RS_FLAG_ANTIALIAS: the adjoint of the antialiased forward (bilinear or
// bicubic); aa = the method whose stretched kernel gives the taps, else 0.
static rs_status bwd_flags(const rs_options& o, rs_method method, int& aa)
{
    if (o.flags & ~RS_FLAG_ANTIALIAS) return RS_ERR_INVALID_ARG;
    aa = 0;
    if (o.flags & RS_FLAG_ANTIALIAS) {
        if (method != RS_BILINEAR && method != RS_BICUBIC) return RS_ERR_INVALID_ARG;
        aa = method == RS_BILINEAR ? M_BILINEAR : M_BICUBIC;
    }
    return RS_OK;
}

extern "C" {

rs_status rs_resize_backward_workspace(const rs_layout* out, const rs_layout* in, rs_method method,
                                       const rs_options* opt, size_t* bytes)
{
    if (!bytes) return RS_ERR_INVALID_ARG;
    const rs_options o = options_or_default(opt);
    int aa = 0;
    rs_status s = bwd_flags(o, method, aa);
    if (s != RS_OK) return s;
    Geom g;
    s = bwd_geom(out, in, method, o, g);
    if (s != RS_OK) return s;
    *bytes = plan_tables(g, method, aa).ws_bytes;
    return RS_OK;
}

rs_status rs_resize_backward(const void* grad_out, const rs_layout* out, void* grad_in, const rs_layout* in,
                             rs_dtype dtype, rs_method method, const rs_options* opt, void* workspace,
                             size_t workspace_bytes, void* stream)
{
    if (dtype != RS_F32) return RS_ERR_UNSUPPORTED;
    const rs_options o = options_or_default(opt);
    int aa = 0;
    rs_status s = bwd_flags(o, method, aa);
    if (s != RS_OK) return s;
    Geom g;
    // make_geom checks pointers, alignment and overlap with src = dX, dst = dY.
    s = make_geom(grad_in, in, grad_out, out, RS_F32, method, o, g);
    if (s != RS_OK) return s;
    BwdPlan p = plan_tables(g, method, aa);
    if (!workspace || workspace_bytes < p.ws_bytes) return RS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return RS_ERR_ALIGNMENT;
    {
        LayoutInfo li, lo;
        classify(in, li);
        classify(out, lo);
        char* ws = static_cast<char*>(workspace);
        if (overlaps(ws, (int64_t)p.ws_bytes, grad_in, li.extent * 4) ||
            overlaps(ws, (int64_t)p.ws_bytes, grad_out, lo.extent * 4))
            return RS_ERR_INVALID_ARG;
    }
    const int KX = p.xK;
    if (KX > 64) return RS_ERR_UNSUPPORTED;   // > 16x upscale along x
    // AUTO: the fused window adjoint where it applies, else the two passes
    // (faster than the tiled kernel at both x2 and x0.5), else the tiled
    // kernel. RS_IMPL_WINDOW / RS_IMPL_STREAM / RS_IMPL_TILED select one
    // (the window adjoint is refused where it does not apply). The two
    // passes use 32-bit offsets within a plane and index the y taps with
    // at most 32 entries.
    AdjWinCfg wcfg;
    const bool window_ok = (o.impl == RS_IMPL_AUTO || o.impl == RS_IMPL_WINDOW) &&
                           adj_window_config(g, p, grad_out, wcfg);
    if (o.impl == RS_IMPL_WINDOW && !window_ok) return RS_ERR_INVALID_ARG;
    if (o.impl == RS_IMPL_PLAIN || o.impl == RS_IMPL_GATHER) return RS_ERR_INVALID_ARG;
    const bool two_pass = !window_ok && o.impl != RS_IMPL_TILED && KX <= 32 && p.yK <= 32 &&
                          (int64_t)g.Ho * g.dst_pitch < (int64_t)INT32_MAX &&
                          (int64_t)g.H * g.src_pitch < (int64_t)INT32_MAX &&
                          (int64_t)g.Ho * g.W * g.C < (int64_t)INT32_MAX;
    AdjCfg cfg;
    if (!window_ok && !two_pass) {
        bool ok = false;
        for (int TH = 32; TH >= 1 && !ok; TH >>= 1) ok = adj_config(g, p, TH, cfg);
        if (!ok) return RS_ERR_UNSUPPORTED;
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    AdjTables tb;
    tb.ylo = reinterpret_cast<int*>(ws + p.off_ylo);
    tb.ycnt = reinterpret_cast<int*>(ws + p.off_ycnt);
    tb.yw = reinterpret_cast<float*>(ws + p.off_yw);
    tb.xlo = reinterpret_cast<int*>(ws + p.off_xlo);
    tb.xcnt = reinterpret_cast<int*>(ws + p.off_xcnt);
    tb.xw = reinterpret_cast<float*>(ws + p.off_xw);
    tb.yK = p.yK;
    tb.xK = p.xK;
    unsigned int* fw = fault_word();
    {
        const TableAxis ya{g.H, g.Ho, tb.yK, (int*)tb.ylo, (int*)tb.ycnt, (float*)tb.yw};
        const TableAxis xa{g.W, g.Wo, tb.xK, (int*)tb.xlo, (int*)tb.xcnt, (float*)tb.xw};
        const int64_t entries = (int64_t)g.H * tb.yK + (int64_t)g.W * tb.xK;
        k_adjoint_tables<<<(unsigned)((entries + 127) / 128), 128, 0, st>>>(ya, xa, method, g.coord, g.a, aa, fw);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    const float* dY = static_cast<const float*>(grad_out);
    float* dX = static_cast<float*>(grad_in);
    if (window_ok) return cuda_status(launch_adj_window(g, p, dY, dX, tb, wcfg, st));
    if (two_pass) {
        float* T = reinterpret_cast<float*>(ws + p.off_t);
        // rows per thread: x pass 8 (4 per iteration) for up to 4 taps, 16 (8
        // per iteration) beyond; y pass 8
        const int rpt = 8;
        const int rpx = KX <= 4 ? 8 : 16;
        const int WC = g.W * g.C;
        const unsigned gx = (unsigned)((WC + kAdjThreads - 1) / kAdjThreads);
        // 16-byte y-pass rows: whole float4s in every T and dX row.
        const bool v4 = WC % 4 == 0 && g.src_pitch % 4 == 0 && reinterpret_cast<uintptr_t>(dX) % 16 == 0 &&
                        (g.planes == 1 || (g.sp.n_stride % 4 == 0 && g.sp.c_stride % 4 == 0));
        const int V = v4 ? 4 : 1;
        const unsigned gy = (unsigned)((WC / V + kAdjThreads - 1) / kAdjThreads);
        for (int p0 = 0; p0 < g.planes; p0 += p.group_planes) {
            const int np = std::min(p.group_planes, g.planes - p0);
            dim3 gxg(gx, (unsigned)((g.Ho + rpx - 1) / rpx), (unsigned)np);
            if (KX <= 4) k_adj_x<4, 4><<<gxg, kAdjThreads, 0, st>>>(g, dY, T, tb, p0, rpx);
            else if (KX <= 8) k_adj_x<8, 8><<<gxg, kAdjThreads, 0, st>>>(g, dY, T, tb, p0, rpx);
            else if (KX <= 16) k_adj_x<16, 8><<<gxg, kAdjThreads, 0, st>>>(g, dY, T, tb, p0, rpx);
            else k_adj_x<32, 8><<<gxg, kAdjThreads, 0, st>>>(g, dY, T, tb, p0, rpx);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
            dim3 gyg(gy, (unsigned)((g.H + rpt - 1) / rpt), (unsigned)np);
            const int KY = p.yK;
            if (v4) {
                if (KY <= 4) k_adj_y<4, 4><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else if (KY <= 8) k_adj_y<8, 4><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else if (KY <= 16) k_adj_y<16, 4><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else k_adj_y<32, 4><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
            } else {
                if (KY <= 4) k_adj_y<4, 1><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else if (KY <= 8) k_adj_y<8, 1><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else if (KY <= 16) k_adj_y<16, 1><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
                else k_adj_y<32, 1><<<gyg, kAdjThreads, 0, st>>>(g, T, dX, tb, p0, rpt);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
        }
        return RS_OK;
    }
    if (KX <= 4) e = launch_adj_c<4>(g, dY, dX, tb, cfg, st);
    else if (KX <= 8) e = launch_adj_c<8>(g, dY, dX, tb, cfg, st);
    else if (KX <= 16) e = launch_adj_c<16>(g, dY, dX, tb, cfg, st);
    else if (KX <= 32) e = launch_adj_c<32>(g, dY, dX, tb, cfg, st);
    else e = launch_adj_c<64>(g, dY, dX, tb, cfg, st);
    return cuda_status(e);
}

}  // extern "C"
