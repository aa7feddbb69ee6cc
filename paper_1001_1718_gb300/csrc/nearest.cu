// Nearest-neighbour kernel: a pure gather, no arithmetic on the samples.
//
// Output element (y, j, c) is source element (ny(y), nx(j), c), with ny / nx
// the exact integer nearest indices (Eq. 2's x1 for the asymmetric map,
// floor(x + 1/2) for the half-pixel map), clamped to the image. Every
// storage type is copied bit for bit.
//
// A block covers a strip of tile_w output elements of rows_per_thread *
// (256 / threads per row) consecutive output rows. Each thread owns 16
// bytes (EV elements) of the strip: their source element offsets are
// computed once into registers. The thread walks rows_per_thread
// consecutive output rows; when a row maps to the same source row as the
// previous one (every other row at x2) the gathered bytes are stored again
// without reloading. Gathers go through the read-only data cache; stores
// are one 16-byte store per thread and row (scalar at unaligned edges).
#include <algorithm>
#include <climits>

#include "capi_internal.h"
#include "rs_common.cuh"

namespace rs {

static constexpr int kNnThreads = 256;
static constexpr int kNnMaxRows = 1024;   // rows of the per-block row table

template <typename T>
__device__ __forceinline__ void put_bits(T* p, uint32_t bits)
{
    if constexpr (sizeof(T) == 1) *reinterpret_cast<uint8_t*>(p) = (uint8_t)bits;
    else if constexpr (sizeof(T) == 2) *reinterpret_cast<uint16_t*>(p) = (uint16_t)bits;
    else *reinterpret_cast<uint32_t*>(p) = bits;
}

template <typename T>
__device__ __forceinline__ uint32_t get_bits(const T* p)
{
    if constexpr (sizeof(T) == 1) return __ldg(reinterpret_cast<const uint8_t*>(p));
    else if constexpr (sizeof(T) == 2) return __ldg(reinterpret_cast<const uint16_t*>(p));
    else return __ldg(reinterpret_cast<const uint32_t*>(p));
}

template <int C, typename T, bool WORDS>
__global__ void __launch_bounds__(kNnThreads)
k_nearest(const Geom g, const T* __restrict__ src, T* __restrict__ dst, int tile_w, int rows_per_thread,
          unsigned int* fault)
{
    constexpr int ES = (int)sizeof(T);
    constexpr int EV = 16 / ES;
    __shared__ int rowtab[kNnMaxRows];
    const int nv = tile_w / EV, vpp = kNnThreads / nv;
    const int tid = threadIdx.x, vx = tid % nv, vy = tid / nv;
    const int plane = blockIdx.z;
    const T* s = src + g.sp.offset(plane);
    T* d = dst + g.dp.offset(plane);
    const int64_t WoC = (int64_t)g.Wo * C;
    const int64_t e0 = (int64_t)blockIdx.x * tile_w + (int64_t)EV * vx;
    const int band = vpp * rows_per_thread;
    const int yb = blockIdx.y * band;
    const int nrows = min(band, g.Ho - yb);
    if (band > kNnMaxRows) {   // uniform; the host bounds the band
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    for (int i = tid; i < nrows; i += kNnThreads)
        rowtab[i] = clampi(nearest_index(yb + i, g.H, g.Ho, g.coord), g.H);
    __syncthreads();

    // Source element offsets of this thread's EV output elements.
    const int cnt = (int)max((int64_t)0, min((int64_t)EV, WoC - e0));
    if (cnt == 0) return;
    int off[EV];
    #pragma unroll
    for (int k = 0; k < EV; ++k) {
        const int64_t e = e0 + min(k, cnt - 1);
        const int j = (int)(e / C), c = (int)(e - (int64_t)j * C);
        off[k] = clampi(nearest_index(j, g.W, g.Wo, g.coord), g.W) * C + c;
    }
    // WORDS: output word q (bytes 4q .. 4q+3 of the thread's 16) is one byte
    // permutation of the two aligned source words wa[q], wb[q]. With the
    // columns upsampled, consecutive output elements step back to the
    // pixel's first channel or forward by one element, so the four source
    // bytes of an output word lie within 4 + 3 bytes of an aligned word.
    int wa[4], wb[4];
    uint32_t sel[4];
    if constexpr (WORDS) {
        bool fit = true;
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            int sb[4];
            #pragma unroll
            for (int i = 0; i < 4; ++i) sb[i] = off[(4 * q + i) / ES] * ES + (4 * q + i) % ES;
            const int lo = min(min(sb[0], sb[1]), min(sb[2], sb[3])) & ~3;
            const int hi = max(max(sb[0], sb[1]), max(sb[2], sb[3])) - lo;
            fit = fit && hi < 8;
            uint32_t m = 0;
            #pragma unroll
            for (int i = 0; i < 4; ++i) m |= (uint32_t)((sb[i] - lo) & 7) << (4 * i);
            sel[q] = m;
            wa[q] = lo >> 2;
            wb[q] = hi >= 4 ? (lo >> 2) + 1 : (lo >> 2);   // never a word without a needed byte
        }
        if (!fit) {   // excluded by the host (columns are upsampled)
            report_fault(fault, FAULT_TILE_SRC_SPAN);
            return;
        }
    }
    uint32_t v[4];
    int last = -1;
    const int i_begin = vy * rows_per_thread;
    const int i_end = min(nrows, i_begin + rows_per_thread);
    for (int i = i_begin; i < i_end; ++i) {
        const int r = rowtab[i];
        if (r != last) {
            const T* row = s + (int64_t)r * g.src_pitch;
            if constexpr (WORDS) {
                const uint32_t* row32 = reinterpret_cast<const uint32_t*>(row);
                #pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = __byte_perm(__ldg(row32 + wa[q]), __ldg(row32 + wb[q]), sel[q]);
            } else {
                uint32_t b[EV];
                #pragma unroll
                for (int k = 0; k < EV; ++k) b[k] = get_bits<T>(row + off[k]);
                if constexpr (ES == 1) {
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[q] = __byte_perm(__byte_perm(b[4 * q], b[4 * q + 1], 0x0040),
                                           __byte_perm(b[4 * q + 2], b[4 * q + 3], 0x0040), 0x5410);
                } else if constexpr (ES == 2) {
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = __byte_perm(b[2 * q], b[2 * q + 1], 0x5410);
                } else {
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = b[q];
                }
            }
            last = r;
        }
        T* out = d + (int64_t)(yb + i) * g.dst_pitch + e0;
        if (cnt == EV && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
            *reinterpret_cast<uint4*>(out) = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
            #pragma unroll
            for (int k = 0; k < EV; ++k) {
                if (k < cnt) {
                    if constexpr (ES == 4) put_bits<T>(out + k, v[k]);
                    else put_bits<T>(out + k, (v[k * ES / 4] >> (8 * ((k * ES) % 4))) & ((1u << (8 * ES)) - 1u));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Staged rows (upsampled columns, 16-byte source rows, 4-byte output rows).
//
// A block owns a strip of 4096 output bytes and a band of output rows and
// walks the band's distinct source rows ("positions") in order. Each
// position's source bytes under the strip are copied into a ring of
// kNnSlots shared-memory rows with 16-byte cp.async copies, kNnSlots - 1
// positions ahead, so DRAM latency is hidden behind the gathers of earlier
// positions (one barrier per position). Thread t owns output words t,
// t + 256, t + 512 and t + 768 of the strip: consecutive lanes read
// neighbouring staged words (no bank conflicts) and each output word is one
// byte permutation of two staged words, stored once per output row that
// maps to the position.
static constexpr int kNnSlots = 4;
static constexpr int kNnStripBytes = 4096;

template <int C, typename T>
__global__ void __launch_bounds__(kNnThreads)
k_nearest_rows(const Geom g, const T* __restrict__ src, T* __restrict__ dst, int band_rows, int span_units,
               unsigned int* fault)
{
    constexpr int ES = (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char nsm[];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;
    const unsigned char* s = reinterpret_cast<const unsigned char*>(src + g.sp.offset(plane));
    unsigned char* d = reinterpret_cast<unsigned char*>(dst + g.dp.offset(plane));
    const int64_t out_row_bytes = (int64_t)g.Wo * C * ES;
    const int64_t b0 = (int64_t)blockIdx.x * kNnStripBytes;
    const int nb = (int)min((int64_t)kNnStripBytes, out_row_bytes - b0);
    const int yb = blockIdx.y * band_rows;
    const int nrows = min(band_rows, g.Ho - yb);
    unsigned char* ring = nsm;                                           // [kNnSlots][span_units * 16]
    int* rowtab = reinterpret_cast<int*>(nsm + (size_t)kNnSlots * span_units * 16);   // [band_rows]
    int* pos_r = rowtab + band_rows;                                     // [band_rows]
    int* pos_i = pos_r + band_rows;                                      // [band_rows + 1]

    // Source bytes under the strip, in whole aligned 16-byte units.
    auto src_byte = [&](int64_t ob) -> int64_t {   // source byte of output byte ob of a row
        const int64_t e = ob / ES;
        const int j = (int)(e / C), c = (int)(e - (int64_t)j * C);
        return ((int64_t)clampi(nearest_index(j, g.W, g.Wo, g.coord), g.W) * C + c) * ES + (ob - e * ES);
    };
    // (whole source pixels: a strip may start or end inside an output pixel)
    const int j_first = (int)(b0 / ES / C), j_last = (int)((b0 + nb - 1) / ES / C);
    const int64_t unit0 = ((int64_t)clampi(nearest_index(j_first, g.W, g.Wo, g.coord), g.W) * C * ES) >> 4;
    const int64_t src_end = ((int64_t)clampi(nearest_index(j_last, g.W, g.Wo, g.coord), g.W) + 1) * C * ES;
    const int units = (int)(((src_end + 15) >> 4) - unit0);
    if (units > span_units || band_rows > kNnMaxRows) {   // uniform; the host sizes both
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }

    // Output word q of this thread: bytes 4 (tid + 256 q) .. +3 of the strip.
    int wa[4], wb[4];
    uint32_t sel[4];
    bool fit = true;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int wo = 4 * (tid + kNnThreads * q);
        int rel[4];
        #pragma unroll
        for (int i = 0; i < 4; ++i)
            rel[i] = (int)(src_byte(b0 + min(wo + i, nb - 1)) - unit0 * 16);
        const int lo = min(min(rel[0], rel[1]), min(rel[2], rel[3])) & ~3;
        const int hi = max(max(rel[0], rel[1]), max(rel[2], rel[3])) - lo;
        fit = fit && hi < 8;
        uint32_t m = 0;
        #pragma unroll
        for (int i = 0; i < 4; ++i) m |= (uint32_t)((rel[i] - lo) & 7) << (4 * i);
        sel[q] = m;
        wa[q] = lo >> 2;
        wb[q] = hi >= 4 ? (lo >> 2) + 1 : (lo >> 2);
    }
    if (!fit) {   // excluded by the host (columns are upsampled)
        report_fault(fault, FAULT_TILE_SRC_SPAN);
    }

    // Source row of every output row of the band, then the positions: runs
    // of equal source rows. Rows never decrease; with rows upsampled every
    // source row between the first and the last is hit, with rows
    // downsampled every output row has its own.
    for (int i = tid; i < nrows; i += kNnThreads) rowtab[i] = clampi(nearest_index(yb + i, g.H, g.Ho, g.coord), g.H);
    __syncthreads();
    const bool rows_up = g.Ho >= g.H;
    const int npos = rows_up ? rowtab[nrows - 1] - rowtab[0] + 1 : nrows;
    if (npos > band_rows) {   // uniform; impossible by the argument above
        if (tid == 0) report_fault(fault, FAULT_TILE_SRC_SPAN);
        return;
    }
    for (int i = tid; i < nrows; i += kNnThreads) {
        if (i == 0 || rowtab[i] != rowtab[i - 1]) {
            const int p = rows_up ? rowtab[i] - rowtab[0] : i;
            pos_r[p] = rowtab[i];
            pos_i[p] = i;
        }
    }
    if (tid == 0) pos_i[npos] = nrows;
    __syncthreads();

    // One commit group per position (empty past the last one).
    auto issue = [&](int p) {
        if (p < npos) {
            const unsigned char* row = s + (int64_t)pos_r[p] * g.src_pitch * ES + unit0 * 16;
            unsigned char* slot = ring + (size_t)(p % kNnSlots) * span_units * 16;
            for (int u = tid; u < units; u += kNnThreads) {
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(slot + u * 16);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(row + u * 16) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    #pragma unroll
    for (int p = 0; p < kNnSlots - 1; ++p) issue(p);

    unsigned char* dband = d + (int64_t)yb * g.dst_pitch * ES + b0;
    const int pitch_b = (int)(g.dst_pitch * ES);
    for (int p = 0; p < npos; ++p) {
        // This thread's copies of position p are done (later groups may
        // still be in flight); the barrier makes every thread's copies
        // visible and ends all reads of the slot that position
        // p + kNnSlots - 1 reuses.
        asm volatile("cp.async.wait_group %0;" ::"n"(kNnSlots - 2) : "memory");
        __syncthreads();
        issue(p + kNnSlots - 1);
        const uint32_t* W = reinterpret_cast<const uint32_t*>(ring + (size_t)(p % kNnSlots) * span_units * 16);
        uint32_t v[4];
        #pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __byte_perm(W[wa[q]], W[wb[q]], sel[q]);
        const int i_end = pos_i[p + 1];
        if (nb == kNnStripBytes) {   // uniform: a full strip, every word in range
            for (int i = pos_i[p]; i < i_end; ++i) {
                uint32_t* out = reinterpret_cast<uint32_t*>(dband + i * pitch_b) + tid;
                #pragma unroll
                for (int q = 0; q < 4; ++q) out[kNnThreads * q] = v[q];
            }
        } else {
            for (int i = pos_i[p]; i < i_end; ++i) {
                unsigned char* out = dband + i * pitch_b;
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int wo = 4 * (tid + kNnThreads * q);
                    if (wo + 4 <= nb) {
                        *reinterpret_cast<uint32_t*>(out + wo) = v[q];
                    } else if (wo < nb) {
                        for (int k = 0; k < nb - wo; ++k) out[wo + k] = (unsigned char)(v[q] >> (8 * k));
                    }
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------

template <int C, typename T>
static void* nn_func(bool words)
{
    return words ? reinterpret_cast<void*>(&k_nearest<C, T, true>) : reinterpret_cast<void*>(&k_nearest<C, T, false>);
}

template <typename T>
static void* nn_func_c(int C, bool words)
{
    switch (C) {
    case 1: return nn_func<1, T>(words);
    case 2: return nn_func<2, T>(words);
    case 3: return nn_func<3, T>(words);
    default: return nn_func<4, T>(words);
    }
}

static void* nn_kernel(int dtype, int C, bool words)
{
    switch (dtype) {
    case DT_U8: return nn_func_c<uint8_t>(C, words);
    case DT_F16: return nn_func_c<__half>(C, words);
    case DT_BF16: return nn_func_c<__nv_bfloat16>(C, words);
    default: return nn_func_c<float>(C, words);
    }
}

// Word gathers need upsampled columns (each output word's bytes within two
// aligned source words) and source rows made of whole aligned 32-bit words.
static bool nn_words(const Geom& g, int dtype, const void* src)
{
    const int64_t es = (int64_t)dtype_size(dtype);
    if (g.Wo < g.W) return false;
    if (reinterpret_cast<uintptr_t>(src) % 4 || (g.src_pitch * es) % 4 || ((int64_t)g.W * g.C * es) % 4) return false;
    if (g.planes > 1 && ((g.sp.n_stride * es) % 4 || (g.sp.c_stride * es) % 4)) return false;
    return true;
}

template <int C, typename T>
static void* nn_rows_func_c() { return reinterpret_cast<void*>(&k_nearest_rows<C, T>); }

template <typename T>
static void* nn_rows_func(int C)
{
    switch (C) {
    case 1: return nn_rows_func_c<1, T>();
    case 2: return nn_rows_func_c<2, T>();
    case 3: return nn_rows_func_c<3, T>();
    default: return nn_rows_func_c<4, T>();
    }
}

static void* nn_rows_kernel(int dtype, int C)
{
    switch (dtype) {
    case DT_U8: return nn_rows_func<uint8_t>(C);
    case DT_F16: return nn_rows_func<__half>(C);
    case DT_BF16: return nn_rows_func<__nv_bfloat16>(C);
    default: return nn_rows_func<float>(C);
    }
}

// The staged-rows kernel: strips of 4096 output bytes (tile_w = 256 x 16 /
// element size), upsampled columns, source rows of whole aligned 16-byte
// units, output rows of whole aligned words, and 32-bit row offsets within
// a band.
static bool nn_rows_ok(const Geom& g, int dtype, const void* src, const void* dst, int tile_w, int band)
{
    const int64_t es = (int64_t)dtype_size(dtype);
    if (tile_w * es != kNnStripBytes || g.Wo < g.W || band < 1 || band > kNnMaxRows) return false;
    if (reinterpret_cast<uintptr_t>(src) % 16 || (g.src_pitch * es) % 16 || ((int64_t)g.W * g.C * es) % 16) return false;
    if (g.planes > 1 && ((g.sp.n_stride * es) % 16 || (g.sp.c_stride * es) % 16)) return false;
    if (reinterpret_cast<uintptr_t>(dst) % 4 || (g.dst_pitch * es) % 4) return false;
    if (g.planes > 1 && ((g.dp.n_stride * es) % 4 || (g.dp.c_stride * es) % 4)) return false;
    return (int64_t)band * g.dst_pitch * es < (int64_t)INT32_MAX;
}

// Upper bound of the 16-byte units a strip of 4096 output bytes reads from
// one source row: its source bytes span at most (4096 / C / es) times the
// coordinate's advance per output, plus one, pixels.
static int nn_rows_units(const Geom& g, int dtype)
{
    const int64_t es = (int64_t)dtype_size(dtype);
    const int64_t px_out = kNnStripBytes / (g.C * es) + 2;
    int64_t an, am;
    coord_advance(g.W, g.Wo, g.coord, an, am);
    const int64_t px_src = (px_out * an + am - 1) / am + 2;
    return (int)((px_src * g.C * es + 15) / 16 + 2);
}

// Default band height of the gather: for the staged-rows kernel, bands that
// leave about two to three blocks per SM (long bands keep each block's
// prefetch ring busy; measured best at 128 rows for an RGB 8192 output),
// between 16 and 256 rows; 32 rows per thread for the per-thread kernel.
int nearest_default_rows(const Geom& g, int dtype)
{
    if (g.Wo < g.W) return 32;
    const int64_t es = (int64_t)dtype_size(dtype);
    const int64_t strips = ((int64_t)g.Wo * g.C * es + kNnStripBytes - 1) / kNnStripBytes;
    const double target = (double)strips * g.Ho * g.planes / (2.5 * num_sms());
    int band = 16;
    while (band < 256 && 2.0 * band <= target) band *= 2;
    return band;
}

bool nearest_config(const Geom& g, int dtype, int tile_w, int rows_per_thread)
{
    const int EV = 16 / (int)dtype_size(dtype);
    if (tile_w < EV || tile_w % EV) return false;
    const int nv = tile_w / EV;
    if (nv > kNnThreads || kNnThreads % nv) return false;
    if (rows_per_thread < 1 || (kNnThreads / nv) * rows_per_thread > kNnMaxRows) return false;
    (void)g;
    return true;
}

cudaError_t launch_nearest(const Geom& g, int dtype, const void* src, void* dst, int tile_w, int rows_per_thread,
                           cudaStream_t st)
{
    if (nn_rows_ok(g, dtype, src, dst, tile_w, rows_per_thread)) {
        const int band = rows_per_thread;
        const int span_units = nn_rows_units(g, dtype);
        const size_t smem = (size_t)kNnSlots * span_units * 16 + sizeof(int) * (3 * (size_t)band + 1);
        if (smem <= max_smem_per_block()) {
            void* func = nn_rows_kernel(dtype, g.C);
            cudaError_t e = prepare_kernel(func, smem, kNnThreads, nullptr);
            if (e != cudaSuccess) return e;
            const int64_t es = (int64_t)dtype_size(dtype);
            dim3 grid((unsigned)(((int64_t)g.Wo * g.C * es + kNnStripBytes - 1) / kNnStripBytes),
                      (unsigned)((g.Ho + band - 1) / band), (unsigned)g.planes);
            unsigned int* fw = fault_word();
            int span = span_units;
            void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, const_cast<int*>(&band), &span, &fw};
            e = cudaLaunchKernel(func, grid, dim3(kNnThreads), args, smem, st);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    const int EV = 16 / (int)dtype_size(dtype);
    const int vpp = kNnThreads / (tile_w / EV);
    const int band = vpp * rows_per_thread;
    dim3 grid((unsigned)(((int64_t)g.Wo * g.C + tile_w - 1) / tile_w), (unsigned)((g.Ho + band - 1) / band),
              (unsigned)g.planes);
    unsigned int* fw = fault_word();
    void* args[] = {const_cast<Geom*>(&g), const_cast<void**>(&src), &dst, &tile_w, &rows_per_thread, &fw};
    cudaError_t e = cudaLaunchKernel(nn_kernel(dtype, g.C, nn_words(g, dtype, src)), grid, dim3(kNnThreads), args, 0, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace rs
