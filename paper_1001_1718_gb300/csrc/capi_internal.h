// Host-side helpers shared by the C ABI translation units.
#pragma once

#include <string>

#include "../../include/resample.h"
#include "rs_internal.h"

namespace rs {

struct LayoutInfo {
    int kind;        // 0 interleaved, 1 planar
    int ci, cp;      // interleaved channels, planes per image
    int64_t extent;  // elements from the base pointer to one past the last element
};

rs_status cuda_status(cudaError_t e);
rs_options options_or_default(const rs_options* opt);
rs_status check_options(const rs_options& o, int method);
rs_status classify(const rs_layout* L, LayoutInfo& info);
bool overlaps(const void* a, int64_t abytes, const void* b, int64_t bbytes);
rs_status geom_from_layouts(const rs_layout* in, const rs_layout* out, int dtype, int method,
                            const rs_options& o, Geom& g, LayoutInfo& li, LayoutInfo& lo);
rs_status make_geom(const void* src, const rs_layout* in, const void* dst, const rs_layout* out,
                    int dtype, int method, const rs_options& o, Geom& g);

// Kernel and configuration for a forward call: explicit options, else the
// tuning cache, else the default (streaming kernel when it fits).
struct KernelChoice {
    int impl;        // RS_IMPL_STREAM, RS_IMPL_TILED, RS_IMPL_GATHER, RS_IMPL_WINDOW or RS_IMPL_REDUCE
    TileCfg tile;
    StreamCfg stream;
    int gather_w, gather_rows;   // RS_IMPL_GATHER: strip width, rows per thread
    WinCfg window;               // RS_IMPL_WINDOW
};
rs_status choose_kernel(const Geom& g, int method, int dtype, const void* src, const rs_options& o,
                        KernelChoice& k);
cudaError_t launch_choice(const Geom& g, int method, int dtype, const void* src, void* dst,
                          const KernelChoice& k, cudaStream_t st);

cudaError_t read_fault(cudaStream_t st, unsigned int* code);

// RS_FLAG_ANTIALIAS forward (backward.cu: the fused window pass with
// computed taps).
rs_status resize_antialias(const Geom& g, int method, int dtype, const void* src, void* dst, const rs_options& o,
                           cudaStream_t st);
// The fused pre-process with RS_FLAG_ANTIALIAS (the antialiased window form).
rs_status resize_normalize_antialias(const Geom& g, int method, int out_dtype, const void* src, void* dst,
                                     const NormOut& no, const rs_options& o, cudaStream_t st);
// RS_IMPL_REDUCE forward (backward.cu: the fused window pass with the
// point taps of Eqs. 1-5 computed in the kernel). reduce_config: whether it
// applies, and its dynamic shared memory.
bool reduce_config(const Geom& g, int method, int dtype, const void* src, size_t* smem);
cudaError_t launch_reduce(const Geom& g, int method, int dtype, const void* src, void* dst, cudaStream_t st);

// Tuning cache entry: kernel (rs_impl) and shape; see autotune.cpp.
struct Tuned {
    int impl, tile_w, tile_h, threads, waves;
};
bool tune_lookup(const std::string& key, Tuned& t);
void tune_store(const std::string& key, const Tuned& t);

}  // namespace rs
