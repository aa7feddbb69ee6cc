// Internal host/device interface of libresample: problem geometry, tile
// configurations and the kernel launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace rs {

enum { COORD_ASYMMETRIC = 0, COORD_HALF_PIXEL = 1, COORD_ALIGN_CORNERS = 2 };

// Advance of the mapped coordinate per output index, as the ratio an / am:
// n / m (asymmetric, half-pixel), (n - 1) / (m - 1) (align-corners; 0 for
// one output). first_tap(j + k - 1) - first_tap(j) <= ceil((k - 1) an / am).
inline void coord_advance(int n, int m, int coord, int64_t& an, int64_t& am)
{
    if (coord == COORD_ALIGN_CORNERS) {
        an = m > 1 ? n - 1 : 0;
        am = m > 1 ? m - 1 : 1;
    } else {
        an = n;
        am = m;
    }
}

// Upper bound of first_tap(j + k - 1) - first_tap(j) + KT over all j: the
// source span of k consecutive outputs with KT taps each.
inline int tap_span_bound(int k, int n, int m, int KT, int coord)
{
    int64_t an, am;
    coord_advance(n, m, coord, an, am);
    const int64_t num = (int64_t)(k - 1) * an;
    return (int)((num + am - 1) / am) + KT;
}
enum { DT_U8 = 0, DT_F16 = 1, DT_BF16 = 2, DT_F32 = 3 };
enum { M_NEAREST = 0, M_BILINEAR = 1, M_BICUBIC = 2 };

// Fault codes recorded in the device fault word.
enum : unsigned int {
    FAULT_NONE = 0,
    FAULT_TILE_SRC_SPAN = 0x101,   // staged source footprint exceeds the smem bound
    FAULT_BWD_SPAN = 0x201,        // backward footprint exceeds the smem bound
    FAULT_BWD_TAPS = 0x202,        // transposed tap count exceeds the table width
    FAULT_BATCH_SPAN = 0x301,      // batched tile footprint exceeds the smem bound
    FAULT_BATCH_INDEX = 0x302,     // batched work index out of range
};

// Addressing of plane p (0 <= p < N * cp) of a batch: planar layouts have cp
// planes per image, interleaved layouts cp = 1.
struct PlaneMap {
    int64_t n_stride, c_stride;
    int cp;
#ifdef __CUDACC__
    __host__ __device__ __forceinline__ int64_t offset(int p) const
    {
        return (int64_t)(p / cp) * n_stride + (int64_t)(p % cp) * c_stride;
    }
#endif
};

// One resampling problem: `planes` images of H x W pixels with C interleaved
// channels (C = 1 for planar data), row pitches in elements.
struct Geom {
    int H, W, Ho, Wo, C;
    int64_t src_pitch, dst_pitch;
    PlaneMap sp, dp;
    int planes;
    int coord;
    float a;
};

// Tile configuration of the tiled forward kernel: tile_w output elements
// (multiple of 4) x tile_h output rows per block of `threads` threads;
// sh_max x swe_max bounds the staged source footprint.
struct TileCfg {
    int tile_w, tile_h, threads;
    int sh_max, swe_max;
    size_t smem;
};

// Configuration of the streaming forward kernel: strips of tile_w output
// elements, chunks of chunk_h output rows, bands of band_h rows per block
// (0 = chosen from occupancy and `waves` blocks per resident slot), an
// rh-row ring (power of two) of horizontally interpolated rows, rs_rows
// staged source rows of swe_max elements; vec = 16-byte loads.
struct StreamCfg {
    int tile_w, chunk_h, band_h, waves;
    int rh, rs_rows, swe_max, vec;
    int band_cap;   // rows of the per-block row-tap table (band_h <= band_cap)
    size_t smem;
};

// Configuration of the register-window kernel (bilinear / bicubic): strips
// of kWinThreads * P output pixels (P per thread, win_pixels), bands of
// band_h output rows (0 = from occupancy and `waves`), source rows staged
// in chunks of `chunk` rows (a multiple of the taps). The rest are
// host-computed bounds every block checks its own strip and band against
// before touching shared memory.
struct WinCfg {
    int chunk, band_h, waves;
    int swe;         // floats per staged FP32 row
    int raw_row;     // bytes per raw staged row
    int band_cap;    // rows of the row-tap tables (band_h <= band_cap)
    int pos_cap;     // source positions of a band
    int tab_off;     // byte offset of the row-tap tables in shared memory
    int raw_off;     // byte offset of the raw ring in shared memory
    int aa_method;   // antialias taps: M_BILINEAR / M_BICUBIC (the stretched kernel)
    int strip;       // antialias taps: output pixels per block (at most the kernel's 128 P)
    size_t smem;
};

// Antialiased resampling with many taps per axis (aa_wide.cu): tiles of 32
// output columns x TH rows; KX / KY = the most taps of an output along x /
// y; fw / nr = the widest source span of a tile's columns / rows; RG =
// source rows staged at a time; s_off = float offset of the staged rows in
// shared memory (after the tap tables).
struct AaWideCfg {
    int KX, KY, TH, RG, fw, nr, method, s_off;
    size_t smem;
};

// Antialiased vertical downscales, vertical pass first (aa_vs.cuh): tiles
// of TW output columns x TH rows; KX = the most x taps of an output; NA =
// register slots of the streamed rows (4, 6 or 8); ve = floats of a finished
// row buffer (the widest tile footprint times the channels, rounded up to 4;
// at most 4 per thread); nr = the most source rows of a band of TH output
// rows; chunk = rows per copy-ring slot; raw_row = bytes per raw ring row.
struct AaVsCfg {
    int KX, TW, TH, NA, ve, nr, chunk, raw_row, method;
    size_t smem;
};

// Output of the fused pre-process (rs_resize_normalize): planar channels,
// channel c of an image at c * c_stride elements from its first element;
// each value is the resampled FP32 value times scale[c] plus bias[c]
// (scale = 1 / std, bias = -mean / std), rounded to the output dtype.
struct NormOut {
    int64_t c_stride;
    float scale[4], bias[4];
};

int method_taps(int method);
size_t dtype_size(int dtype);

// Maximum dynamic shared memory a block may use on this device.
size_t max_smem_per_block();
int num_sms();
// GPU name, compute capability and CUDA runtime version of the current
// device, as one token (tuning-cache keys).
const std::string& device_tag();
// Raises func's dynamic shared-memory limit to at least smem bytes and, if
// per_sm is given, returns its resident blocks per SM at `threads` threads
// and smem bytes; both driver queries are cached per device and kernel.
cudaError_t prepare_kernel(const void* func, size_t smem, int threads, int* per_sm);

// Fault word of the current device (a static __device__ word resolved by
// cudaGetSymbolAddress), or nullptr if it cannot be resolved.
unsigned int* fault_word();

// Completes cfg (sh_max, swe_max, smem) for the problem; false if the
// configuration is malformed or does not fit in shared memory.
bool tiled_config(const Geom& g, int method, TileCfg& cfg);
TileCfg tiled_default(const Geom& g, int method);

cudaError_t launch_tiled(const Geom& g, int method, int dtype, const void* src, void* dst,
                         const TileCfg& cfg, cudaStream_t st);
bool stream_config(const Geom& g, int method, int dtype, const void* src, StreamCfg& c);
StreamCfg stream_default(const Geom& g, int method, int dtype, const void* src);
cudaError_t launch_stream(const Geom& g, int method, int dtype, const void* src, void* dst, StreamCfg c,
                          cudaStream_t st);
// Register-window kernel: pixels per thread, whether the exact-x2 form
// applies (asymmetric map, both axes exactly doubled), configuration (false
// if malformed or beyond shared memory; allow_x2 = false sizes the general
// form even where the exact-x2 one applies) and launch.
int win_pixels(int C, int dtype, bool x2);
bool win_is_x2(const Geom& g);
bool win_config(const Geom& g, int method, int dtype, WinCfg& c, bool allow_x2 = true);
cudaError_t launch_win(const Geom& g, int method, int dtype, const void* src, void* dst, WinCfg c, cudaStream_t st);
// Antialiased resampling (RS_FLAG_ANTIALIAS) on the general window form:
// the most taps any output has on either axis (antialias_taps), the tap
// capacity K (4 or 8; 0: too many), configuration and launch (out_dtype /
// no: the fused pre-process's normalised planar output when norm is set).
int antialias_taps(const Geom& g, int method);
bool win_config_aa(const Geom& g, int method, int dtype, int K, WinCfg& c);
cudaError_t launch_win_aa(const Geom& g, int method, int dtype, const void* src, void* dst, int K, WinCfg c,
                          cudaStream_t st);
cudaError_t launch_win_aa_norm(const Geom& g, int method, int out_dtype, const void* src, void* dst, int K, WinCfg c,
                               const NormOut& no, cudaStream_t st);
// Antialias taps beyond the window forms (aa_wide.cu): false where a
// tile's footprint cannot fit in shared memory.
bool aa_wide_config(const Geom& g, int method, AaWideCfg& c);
// The vertical-first form (aa_vs.cuh): false where it does not apply (a
// vertical upscale, too wide a footprint, too many overlapping output rows).
bool aa_vs_config(const Geom& g, int method, int dtype, AaVsCfg& c);
cudaError_t launch_aa_vs(const Geom& g, int dtype, const void* src, void* dst, const AaVsCfg& c, cudaStream_t st);
cudaError_t launch_aa_vs_norm(const Geom& g, int out_dtype, const void* src, void* dst, const AaVsCfg& c,
                              const NormOut& no, cudaStream_t st);
cudaError_t launch_aa_wide(const Geom& g, int dtype, const void* src, void* dst, const AaWideCfg& c, cudaStream_t st);
cudaError_t launch_aa_wide_norm(const Geom& g, int out_dtype, const void* src, void* dst, const AaWideCfg& c,
                                const NormOut& no, cudaStream_t st);
// The fused pre-process on the window kernels: uint8 interleaved source
// (g describes it; g.dp / g.dst_pitch the output images and rows),
// normalised planar output of out_dtype (DT_F16, DT_BF16 or DT_F32).
cudaError_t launch_win_norm(const Geom& g, int method, int out_dtype, const void* src, void* dst, WinCfg c,
                            const NormOut& no, cudaStream_t st);
bool nearest_config(const Geom& g, int dtype, int tile_w, int rows_per_thread);
int nearest_default_rows(const Geom& g, int dtype);
cudaError_t launch_nearest(const Geom& g, int dtype, const void* src, void* dst, int tile_w, int rows_per_thread,
                           cudaStream_t st);
cudaError_t launch_plain(const Geom& g, int method, int dtype, const void* src, void* dst,
                         int bw, int bh, cudaStream_t st);

}  // namespace rs
