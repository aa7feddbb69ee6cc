/*
 * resample.h -- C ABI of the GB300 image-resampling library (libresample.so).
 *
 * The library resamples 2-D images by nearest-neighbour, bilinear or bicubic
 * interpolation on one GPU. The operation is the paper's image resizing
 * (Sec. II.B, Eqs. 1-5): every output pixel (x_f, y_f) maps to the source
 * point x_p = x_f / scale, y_p = y_f / scale (Eq. 1), takes the neighbours
 * int(x_p), int(x_p) + 1 (Eqs. 2-3) with fractional offsets (Eq. 4) and
 * blends them (Eq. 5). The paper names nearest-neighbour and bicubic
 * interpolation without defining them; the library defines them as follows.
 *
 *   Per axis, for output index j of m outputs from n source samples:
 *   - scale is m / n, taken from the sizes, so x = j * n / m exactly
 *     (RS_COORD_ASYMMETRIC, the paper's Eq. 1); RS_COORD_HALF_PIXEL maps
 *     pixel centres instead: x = (j + 1/2) * n / m - 1/2;
 *     RS_COORD_ALIGN_CORNERS (an extension) pins the first and last
 *     samples together: x = j * (n - 1) / (m - 1), x = 0 when m = 1;
 *   - i0 = floor(x), t = x - i0 (Eqs. 2-4);
 *   - RS_NEAREST: sample i0 (asymmetric) or floor(x + 1/2) (half-pixel,
 *     align-corners);
 *     RS_BILINEAR: samples i0, i0+1, weights 1-t, t (Eq. 5);
 *     RS_BICUBIC: samples i0-1 .. i0+2, weights K(t+1), K(t), K(1-t), K(2-t)
 *     with Keys' cubic convolution kernel K of parameter a (default -1/2);
 *   - every sample index is clamped to [0, n-1] (edge replicate).
 *   The 2-D result is the product of the two axes' weights summed over the
 *   taps, per channel. Arithmetic is FP32 (weights and accumulation) for
 *   every storage type. Stores round to nearest even; uint8 stores clamp to
 *   [0, 255] first.
 *
 * Conventions shared by every entry point:
 *   - All image pointers are DEVICE pointers the caller owns. The library
 *     never allocates, frees or synchronises caller memory or streams.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream). RS_OK means the work was enqueued.
 *   - Arguments are validated on the host before anything is launched. On
 *     any error status nothing is launched and no output is written.
 *   - Sizes: 1 <= H, W, Ho, Wo <= 65535. Strides are in ELEMENTS.
 *   - Inputs and outputs must not overlap (RS_ERR_INVALID_ARG).
 *   - Thread-safe for distinct streams. Calls on one stream run in order.
 *   - RS_ERR_CUDA reports a launch or runtime error; rs_last_cuda_error()
 *     returns its CUDA error code for the calling thread.
 */
#ifndef RESAMPLE_H
#define RESAMPLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = 1,   /* null pointer, size out of range, overlap, bad stride */
    RS_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
    RS_ERR_ALIGNMENT = 3,     /* pointer not aligned to its element size */
    RS_ERR_WORKSPACE = 4,     /* workspace null or smaller than required */
    RS_ERR_CUDA = 5           /* CUDA launch / runtime error */
} rs_status;

typedef enum { RS_U8 = 0, RS_F16 = 1, RS_BF16 = 2, RS_F32 = 3 } rs_dtype;
typedef enum { RS_NEAREST = 0, RS_BILINEAR = 1, RS_BICUBIC = 2 } rs_method;
typedef enum { RS_COORD_ASYMMETRIC = 0, RS_COORD_HALF_PIXEL = 1, RS_COORD_ALIGN_CORNERS = 2 } rs_coord;

/* Kernel selection.
 * AUTO   = the tuned (or default) kernel for the problem: GATHER for
 *          RS_NEAREST; for bilinear / bicubic REDUCE on RS_F32 vertical
 *          downscales to at least 1/4 (outputs >= 2^20 elements), WINDOW on
 *          vertical upscales and uint8 outputs of at least 2^22 elements,
 *          where its footprint fits in shared memory; else STREAM, else
 *          TILED. rs_autotune replaces this choice for a problem it has
 *          timed.
 * WINDOW = bilinear / bicubic, blocks of 128 threads, one per (strip of
 *          output pixels, band of output rows, plane). Source rows are
 *          copied with 16-byte cp.async in chunks of tile_h rows (a
 *          multiple of the taps: 2 bilinear, 4 bicubic) two chunks ahead;
 *          each thread interpolates every source row its pixels' taps reach
 *          horizontally once, keeps the last 2 or 4 such rows in registers,
 *          and blends each output row from them (no shared-memory traffic
 *          per output row). Two forms:
 *          exact x2 (asymmetric map, both axes exactly doubled): a thread
 *          owns P consecutive output pixels (P * C * size >= 8 bytes where
 *          the row allows), reads its footprint straight from the copied
 *          bytes and stores its run with packed 4- to 16-byte stores; the
 *          even outputs are copies, the odd ones the midpoint weights;
 *          general ratios: a thread owns P pixels 32 apart (strips of
 *          128 P pixels, P = 2 to 8 by channels and dtype) over source rows
 *          converted to channel-planar FP32 in shared memory.
 *          waves = blocks per resident block slot (sets the band height).
 * STREAM = one block per (column strip, band of rows), walking down the band
 *          in chunks; every source row is staged and horizontally
 *          interpolated once per strip; loads of the next chunk are issued
 *          while the current one computes. tile_w = strip width in output
 *          elements, tile_h = rows per chunk, waves = blocks per resident
 *          block slot (sets the band height).
 * TILED  = one block per output tile of tile_w elements x tile_h rows with
 *          `threads` threads; the footprint and halo are staged per tile.
 * GATHER = RS_NEAREST only (AUTO's choice for it): a bit-exact gather.
 *          tile_w = 256 x 16 bytes (default) with upsampled columns and
 *          16-byte-aligned source rows: a block walks the distinct source
 *          rows of a band of tile_h output rows (default: 16..256 rows, about
 *          two to three blocks per SM), staging each
 *          one's bytes under its 4096-byte strip in shared memory three
 *          rows ahead, and writes every output row that maps to it.
 *          Otherwise each thread copies 16 bytes of a strip of tile_w output
 *          elements over tile_h consecutive output rows, reusing a gathered
 *          row for the next output row when both map to the same source row.
 * REDUCE = RS_F32 bilinear / bicubic with source rows of whole aligned
 *          16-byte units (pointer, pitch and W*C multiples of 4 elements):
 *          the register window in its transposed roles (the backward's fused
 *          kernel with the taps of Eqs. 1-5 computed in the kernel). Each
 *          thread owns 2 output elements (strided by 256) of a 512-element
 *          strip for a band of output rows; the source rows the band's taps
 *          reach are copied with 16-byte cp.async into a three-slot ring and
 *          horizontally interpolated at the thread's columns into a register
 *          window; every output row whose first tap is the window's first
 *          row is blended from registers. Taps that clamp onto the same
 *          edge column are merged (their weights summed), so sums at the
 *          left and right edges may round differently from the other
 *          kernels. Any scale; tile_w / tile_h / threads / waves must be 0.
 * PLAIN  = one thread per output pixel reading its taps from global memory,
 *          thread blocks of tile_w x tile_h threads (default 32 x 4): the
 *          paper's kernel (Sec. III.A, Eq. 6), kept as the comparison row. */
typedef enum { RS_IMPL_AUTO = 0, RS_IMPL_TILED = 1, RS_IMPL_PLAIN = 2, RS_IMPL_STREAM = 3,
               RS_IMPL_GATHER = 4, RS_IMPL_WINDOW = 5, RS_IMPL_REDUCE = 6 } rs_impl;

/* Option flags.
 * RS_FLAG_ANTIALIAS - an extension beyond the paper's point sampling: the
 *   bilinear (triangle) or bicubic (Keys, cubic_a) kernel is stretched by
 *   the downscale factor f = max(n / m, 1) of each axis, so an output
 *   averages the source footprint it covers: output j has centre
 *   c = (j + 1/2) n / m, taps i = floor(c - R f + 1/2) .. floor(c + R f +
 *   1/2) - 1 (R = 1 bilinear, 2 bicubic) cut to [0, n), weights
 *   K((i + 1/2 - c) / f) renormalised to sum 1 (no edge replication; the
 *   coord option does not apply). Every storage dtype, any downscale whose
 *   tile footprint fits in shared memory (about 1/64 and above). Kernels:
 *   RS_F32 with 16-byte source rows and at most 8 taps per axis: REDUCE's
 *   fused pass with these taps; otherwise, up to 8 taps per axis (bilinear
 *   down to 1/4, bicubic to 1/2), WINDOW's general form with these taps
 *   (impl RS_IMPL_WINDOW selects it and refuses more taps); beyond that, on
 *   vertical downscales (output rows <= source rows), a vertical-first
 *   streaming kernel (each tile's source rows copied once through a
 *   shared-memory ring, the vertical sums kept in registers, the finished
 *   rows blended horizontally; impl RS_IMPL_STREAM selects it, and refuses
 *   vertical upscales), else, or with impl RS_IMPL_TILED, a tiled kernel
 *   that holds any number of taps (tiles of 32 output columns: the tile's
 *   footprint rows are interpolated horizontally into shared memory, then
 *   blended).
 *   RS_NEAREST: RS_ERR_INVALID_ARG. Also for rs_resize_normalize,
 *   rs_resize_backward (the adjoint of this map) and the batch. */
#define RS_FLAG_ANTIALIAS 1

typedef struct {
    int32_t coord;      /* rs_coord; default RS_COORD_ASYMMETRIC */
    float cubic_a;      /* Keys parameter a for RS_BICUBIC; default -0.5 */
    int32_t impl;       /* rs_impl; default RS_IMPL_AUTO */
    int32_t tile_w;     /* 0 = default. PLAIN: threads per block along x.
                           TILED: output elements per tile row (multiple of 4*32). */
    int32_t tile_h;     /* 0 = default. PLAIN: threads along y. TILED: output rows per tile. */
    int32_t threads;    /* 0 = default. TILED: threads per block (128 or 256). */
    int32_t waves;      /* 0 = default. STREAM: blocks per resident block slot. */
    int32_t flags;      /* RS_FLAG_* bits; 0 = none */
} rs_options;

/* Fills *opt with the defaults listed above. */
void rs_options_init(rs_options* opt);

/*
 * Memory layout of a batch of N images of C channels, H rows, W columns.
 * Element (n, c, y, x) is at n*n_stride + c*c_stride + y*row_pitch + x*px_stride.
 * Two layouts are accepted:
 *   interleaved (NHWC / HWC): px_stride == C, c_stride == 1, C <= 4;
 *   planar (NCHW):            px_stride == 1 (C planes of H x W each).
 * For C == 1 both readings coincide. row_pitch >= W * px_stride.
 */
typedef struct {
    int32_t N, C, H, W;
    int64_t n_stride, c_stride, row_pitch, px_stride;
} rs_layout;

/* Tightly packed layouts: interleaved HWC (n_stride = H*W*C) and planar NCHW. */
rs_layout rs_layout_hwc(int32_t N, int32_t H, int32_t W, int32_t C);
rs_layout rs_layout_nchw(int32_t N, int32_t C, int32_t H, int32_t W);

const char* rs_status_string(rs_status s);
const char* rs_version(void);
/* CUDA error code (cudaError_t) behind the calling thread's last RS_ERR_CUDA. */
int rs_last_cuda_error(void);

/*
 * Diagnostic: synchronises `stream`, then reads and clears the current
 * device's fault word. A kernel that finds an internal bound violated (a
 * staged footprint larger than its shared-memory bound, a work index out of
 * range) records a nonzero code there and skips the access instead of
 * faulting. 0 means no kernel has reported anything since the last read.
 */
rs_status rs_debug_fault(void* stream, uint32_t* code);

/*
 * Resize one tightly packed HWC image (Sec. II.B, Eqs. 1-5): src is H x W x C
 * of `dtype`, dst is Ho x Wo x C of the same dtype, 1 <= C <= 4. Asymmetric
 * map (Eq. 1), a = -1/2: rs_resize_ex with the default options, so the
 * kernel is RS_IMPL_AUTO's choice.
 */
rs_status rs_resize(const void* src, int H, int W, int C, rs_dtype dtype,
                    void* dst, int Ho, int Wo, rs_method method, void* stream);

/*
 * General form: N images of any accepted layout (in / out must have the same
 * N, C and layout kind; strides may differ). opt may be NULL (defaults).
 */
rs_status rs_resize_ex(const void* src, const rs_layout* in, void* dst,
                       const rs_layout* out, rs_dtype dtype, rs_method method,
                       const rs_options* opt, void* stream);

/*
 * Fused serving pre-process (an extension of Sec. II.B, Eqs. 1-5): resample
 * a uint8 interleaved batch (in: N images of H x W x C, C <= 4, any pitches)
 * bilinearly or bicubically, normalise every channel, y = (x - mean[c]) /
 * stddev[c], and store it planar (out: N x C x Ho x Wo, px_stride 1; for C = 1
 * either layout) as RS_F16, RS_BF16 or RS_F32, rounded to nearest even --
 * one pass over the source and one over the output, where a resize followed
 * by a separate normalise-and-transpose pass reads and writes the image
 * twice and rounds it to uint8 in between. The resampled value stays FP32
 * (it is never rounded to uint8); the normalisation is one FP32 fused
 * multiply-add per element with scale 1 / stddev[c] and bias -mean[c] /
 * stddev[c]. mean, stddev: C host floats each (finite, stddev nonzero). Options: coord and
 * cubic_a as for rs_resize_ex; impl RS_IMPL_AUTO or RS_IMPL_WINDOW (the
 * register-window kernel; tile_h = staged rows per chunk, waves); flags 0
 * or RS_FLAG_ANTIALIAS (the antialiased window form up to 8 taps per axis;
 * beyond that, unless impl is RS_IMPL_WINDOW, the vertical-first streaming
 * kernel on vertical downscales, else the many-tap tiled kernel; tile_h
 * must be 0). RS_NEAREST returns RS_ERR_UNSUPPORTED, and so does a point-
 * sampled downscale whose staged footprint exceeds shared memory (about
 * 1/5 and below; RS_FLAG_ANTIALIAS is the filter for such downscales).
 */
rs_status rs_resize_normalize(const void* src, const rs_layout* in, void* dst, const rs_layout* out,
                              rs_dtype out_dtype, rs_method method, const float* mean, const float* stddev,
                              const rs_options* opt, void* stream);

/*
 * Backward (adjoint) of rs_resize_ex for RS_F32: grad_in = A^T grad_out,
 * where A is the linear map the forward applies (per axis, the transpose of
 * the interpolation weights, summed over the clamped taps). Computed in
 * gather form: every input sample sums, in a fixed order, the output
 * samples whose taps name it, so results are deterministic (no atomics).
 * grad_in is OVERWRITTEN. `workspace` is a device buffer of at least the
 * size rs_resize_backward_workspace() reports: the per-axis transposed weight
 * tables and an FP32 intermediate (the x-transposed rows of a group of
 * planes, at most ~256 MB); it is written by the call and may be reused after
 * the call's work on `stream` has finished. Kernels (opt->impl):
 *   RS_IMPL_AUTO   - WINDOW where it applies, else STREAM, else TILED;
 *   RS_IMPL_WINDOW - one fused pass: each thread keeps the x-transposed
 *                    dY rows its y taps need in registers (at most 8
 *                    transposed taps per axis, dY rows of whole aligned
 *                    16-byte units; RS_ERR_INVALID_ARG otherwise); same
 *                    results as STREAM;
 *   RS_IMPL_STREAM - two passes through the intermediate (x, then y);
 *   RS_IMPL_TILED  - one tiled pass through shared memory.
 * Only the tables (and, for STREAM, the intermediate) of the workspace are
 * used. opt->flags: 0, or RS_FLAG_ANTIALIAS for the adjoint of the
 * antialiased forward (bilinear / bicubic; the tables then hold the
 * transposed antialias weights, and the same three kernels apply); pass the
 * same opt to rs_resize_backward_workspace. Other flags, and
 * RS_FLAG_ANTIALIAS with RS_NEAREST: RS_ERR_INVALID_ARG.
 */
rs_status rs_resize_backward_workspace(const rs_layout* out, const rs_layout* in,
                                       rs_method method, const rs_options* opt,
                                       size_t* bytes);
rs_status rs_resize_backward(const void* grad_out, const rs_layout* out,
                             void* grad_in, const rs_layout* in, rs_dtype dtype,
                             rs_method method, const rs_options* opt,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * Ragged batch: n independent images, each with its own size, scale, channel
 * count (interleaved, 1..4) and method, resampled by ONE persistent kernel
 * launch that walks a work list of output tiles. Host array of descriptors;
 * pitches in elements. All images share `dtype` and the options' coord and a.
 */
typedef struct {
    const void* src;
    void* dst;
    int32_t H, W, C, Ho, Wo;
    int32_t method;            /* rs_method */
    int64_t src_pitch, dst_pitch;
} rs_image_desc;

/*
 * Batch options (rs_options): coord and cubic_a apply to every image.
 * impl = RS_IMPL_AUTO: bilinear / bicubic images whose source footprint
 *   fits run as register-window items (bands of 256 output rows, source
 *   rows staged 8 at a time, else 4), the rest as tiles; when
 *   rs_autotune_batched has tuned this batch (same sizes, methods, pitches,
 *   dtype, count and coord) its shape is used instead. An explicit tile_w /
 *   tile_h / threads tiles every image.
 * impl = RS_IMPL_WINDOW: window items with band = tile_w output rows
 *   (1..256, 0 = 256) and chunk = tile_h staged rows (4..32, a multiple of
 *   the taps, 0 = 8 else 4);
 *   images that do not fit are tiled.
 * impl = RS_IMPL_TILED: every image as tiles of tile_w elements (0 = 512)
 *   x at most tile_h rows (0 = 32) with `threads` threads (0 = 256).
 * Other impl values return RS_ERR_INVALID_ARG.
 * flags = RS_FLAG_ANTIALIAS: every image with the antialias taps (bilinear
 *   / bicubic only; a nearest image returns RS_ERR_INVALID_ARG): window
 *   items up to 8 taps per axis, the many-tap tiled kernel's tiles beyond
 *   (and for every image under RS_IMPL_TILED). Other flags:
 *   RS_ERR_INVALID_ARG.
 */

/* Device workspace bytes rs_resize_batched needs for these descriptors. */
rs_status rs_resize_batched_workspace(const rs_image_desc* d, int n, rs_dtype dtype,
                                      size_t* bytes);
/* Uploads the work list into `workspace` (async on `stream`) and launches. */
rs_status rs_resize_batched(const rs_image_desc* d, int n, rs_dtype dtype,
                            void* workspace, size_t workspace_bytes,
                            const rs_options* opt, void* stream);

/*
 * Ragged batch without any allocation, for callers that cannot obtain
 * device memory for a workspace: code under an allocator that owns all
 * device memory (a framework's caching pool, a fixed memory budget),
 * serving paths that forbid allocation after start-up because cudaMalloc
 * can block or fail, and plugin hosts that only hand out input and output
 * buffers. The paper has no counterpart; this is a deployment variant of
 * rs_resize_batched with the same arguments minus the workspace, and the
 * same results.
 *
 * The work list goes into a fixed array of device memory declared inside
 * the library (static __device__, RS_NOALLOC_MAX_IMAGES descriptors, about
 * 650 KB); every GPU that loads the library holds it until the process
 * exits. Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 * routine is called.
 *   - n > RS_NOALLOC_MAX_IMAGES returns RS_ERR_WORKSPACE, before any work.
 *   - The first call on a device looks up the array's device address (with
 *     that device current).
 *   - Every call shares the one array and overwrites it (nothing in it needs
 *     to start at zero: each call writes all it reads). Calls whose work
 *     overlaps on the GPU (for example on two streams at once) race on it;
 *     calls on one stream run in order and are safe.
 *   - The descriptors are copied from host staging memory on `stream` before
 *     the launch (the call returns once they are staged); src / dst stay
 *     owned by the caller as in rs_resize_batched. While `stream` is being
 *     captured the call returns RS_ERR_UNSUPPORTED and does nothing: the next
 *     call refills the staging memory a captured copy would read. Replayable
 *     batches are rs_batched_plan_*'s job.
 */
#define RS_NOALLOC_MAX_IMAGES 4096
rs_status rs_resize_batched_noalloc(const rs_image_desc* d, int n, rs_dtype dtype,
                                    const rs_options* opt, void* stream);

/*
 * Replayable batch: the work list is uploaded once and the persistent launch
 * is recorded as a CUDA graph; each rs_batched_plan_launch replays it on a
 * stream. The plan refers to the descriptors' src / dst buffers and to
 * `workspace`, which must stay valid until rs_batched_plan_destroy.
 */
typedef struct rs_batched_plan rs_batched_plan;
rs_status rs_batched_plan_create(const rs_image_desc* d, int n, rs_dtype dtype,
                                 void* workspace, size_t workspace_bytes,
                                 const rs_options* opt, void* stream,
                                 rs_batched_plan** plan);
rs_status rs_batched_plan_launch(rs_batched_plan* plan, void* stream);
/* Kernel launches one replay makes: one persistent launch per non-empty class
 * (window items by method, channel count and footprint tier; tiles). */
rs_status rs_batched_plan_kernels(const rs_batched_plan* plan, int32_t* kernels);
rs_status rs_batched_plan_destroy(rs_batched_plan* plan);

/*
 * Autotuner. A configuration is a kernel and its shape: WINDOW chunk height
 * tile_h with `waves` blocks per resident slot; STREAM strip width tile_w x
 * chunk height tile_h with `waves`; TILED tile_w elements x tile_h rows with
 * `threads` threads; GATHER (nearest) strip width x rows; REDUCE (FP32,
 * no shape).
 * rs_autotune times every candidate configuration on the caller's buffers
 * (dst is overwritten; the stream is synchronised while it runs) and stores
 * the fastest in the in-process cache, keyed by GPU, dtype, method, channel
 * layout and scale class; later RS_IMPL_AUTO calls with that key use it.
 * The cache can be saved to and loaded from a text file.
 */
typedef struct {
    int32_t impl;       /* RS_IMPL_WINDOW, RS_IMPL_REDUCE, RS_IMPL_STREAM, RS_IMPL_TILED or RS_IMPL_GATHER */
    int32_t tile_w, tile_h, threads, waves;
    float best_us;      /* measured time of the chosen configuration */
    float default_us;   /* measured time of the default configuration */
    int32_t candidates; /* number of configurations timed */
} rs_tile_config;

rs_status rs_autotune(const void* src, const rs_layout* in, void* dst,
                      const rs_layout* out, rs_dtype dtype, rs_method method,
                      const rs_options* opt, void* stream, rs_tile_config* best);
/*
 * Batch autotuner: runs the batch (dst buffers are written; the stream is
 * synchronised while it runs) for each item shape in a small sweep -- band
 * heights 32..256 and chunk heights 8 / 4 of the window items, and all
 * tiles -- and stores the fastest in the same cache under a key made of the
 * GPU, dtype, image count, coord and a hash of every descriptor's sizes,
 * channels, method and pitches. Later RS_IMPL_AUTO batch calls (direct or
 * plans) with that key use it; rs_resize_batched_noalloc does not consult
 * the cache. best: impl (RS_IMPL_WINDOW or RS_IMPL_TILED), tile_w = band
 * rows, tile_h = chunk rows (0 = 8 else 4), the chosen and the default
 * shape's mean time per batch launch, and the number of shapes timed.
 * `workspace` as for rs_resize_batched.
 */
rs_status rs_autotune_batched(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace,
                              size_t workspace_bytes, const rs_options* opt, void* stream,
                              rs_tile_config* best);
rs_status rs_tune_cache_save(const char* path);
rs_status rs_tune_cache_load(const char* path);
void rs_tune_cache_clear(void);
/* The configuration RS_IMPL_AUTO would use for this problem (cached or default). */
rs_status rs_tile_config_for(const rs_layout* in, const rs_layout* out, rs_dtype dtype,
                             rs_method method, const rs_options* opt, rs_tile_config* cfg);

#ifdef __cplusplus
}
#endif

#endif /* RESAMPLE_H */
