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
