// Tiled separable forward kernel: one thread block per output tile (the
// tile's work is tile_body in tile_body.cuh) and the host-side tile
// configuration.
#include "tile_body.cuh"

namespace rs {

template <int KT, int C, typename T>
__global__ void __launch_bounds__(256)
k_tiled(const Geom g, const T* __restrict__ src, T* __restrict__ dst, const TileCfg cfg,
        unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    const int plane = blockIdx.z;
    tile_body<KT, C, T>(g, src + g.sp.offset(plane), dst + g.dp.offset(plane), cfg, blockIdx.x,
                        blockIdx.y, sm, fault);
}

// ---------------------------------------------------------------------------
// Host side

bool tiled_config(const Geom& g, int method, TileCfg& cfg)
{
    const int KT = method_taps(method);
    if (cfg.tile_w < 4 || (cfg.tile_w & 3) || cfg.tile_h < 1) return false;
    if (cfg.threads != 128 && cfg.threads != 256) return false;
    const int nq = cfg.tile_w / 4;
    if (nq > cfg.threads || cfg.threads % nq) return false;
    const int kpx = (cfg.tile_w + g.C - 1) / g.C + 1;   // pixels a tile row can touch
    cfg.sh_max = tap_span_bound(cfg.tile_h, g.H, g.Ho, KT, g.coord);
    int swe = tap_span_bound(kpx, g.W, g.Wo, KT, g.coord) * g.C;
    cfg.swe_max = (swe + 3) & ~3;
    cfg.smem = sizeof(float) * ((size_t)cfg.sh_max * cfg.swe_max + (size_t)cfg.sh_max * cfg.tile_w +
                                (size_t)cfg.tile_h * KT) +
               sizeof(int) * (size_t)cfg.tile_h;
    return cfg.smem <= max_smem_per_block();
}

TileCfg tiled_default(const Geom& g, int method)
{
    // 256 threads, 512 output elements per tile row; the tallest tile (<= 32
    // rows) whose footprint fits in ~72 KB (three blocks per SM), else the
    // smallest that fits at all.
    static const int widths[] = {512, 256, 128};
    for (int wi = 0; wi < 3; ++wi) {
        for (int th = 32; th >= 1; th >>= 1) {
            TileCfg c{widths[wi], th, 256, 0, 0, 0};
            if (tiled_config(g, method, c) && c.smem <= 72 * 1024) return c;
        }
    }
    for (int wi = 0; wi < 3; ++wi) {
        for (int th = 32; th >= 1; th >>= 1) {
            TileCfg c{widths[wi], th, 256, 0, 0, 0};
            if (tiled_config(g, method, c)) return c;
        }
    }
    return TileCfg{0, 0, 0, 0, 0, 0};
}

template <int KT, int C, typename T>
static cudaError_t launch_t(const Geom& g, const void* src, void* dst, const TileCfg& cfg,
                            cudaStream_t st)
{
    auto kern = k_tiled<KT, C, T>;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), cfg.smem, cfg.threads, nullptr);
    if (e != cudaSuccess) return e;
    const int64_t WoC = (int64_t)g.Wo * C;
    dim3 grid((unsigned)((WoC + cfg.tile_w - 1) / cfg.tile_w),
              (unsigned)((g.Ho + cfg.tile_h - 1) / cfg.tile_h), (unsigned)g.planes);
    kern<<<grid, cfg.threads, cfg.smem, st>>>(g, static_cast<const T*>(src), static_cast<T*>(dst),
                                              cfg, fault_word());
    return cudaGetLastError();
}

template <int KT, typename T>
static cudaError_t launch_c(const Geom& g, const void* src, void* dst, const TileCfg& cfg,
                            cudaStream_t st)
{
    switch (g.C) {
    case 1: return launch_t<KT, 1, T>(g, src, dst, cfg, st);
    case 2: return launch_t<KT, 2, T>(g, src, dst, cfg, st);
    case 3: return launch_t<KT, 3, T>(g, src, dst, cfg, st);
    case 4: return launch_t<KT, 4, T>(g, src, dst, cfg, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_m(const Geom& g, int method, const void* src, void* dst,
                            const TileCfg& cfg, cudaStream_t st)
{
    switch (method) {
    case M_NEAREST: return launch_c<1, T>(g, src, dst, cfg, st);
    case M_BILINEAR: return launch_c<2, T>(g, src, dst, cfg, st);
    case M_BICUBIC: return launch_c<4, T>(g, src, dst, cfg, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tiled(const Geom& g, int method, int dtype, const void* src, void* dst,
                         const TileCfg& cfg, cudaStream_t st)
{
    switch (dtype) {
    case DT_U8: return launch_m<uint8_t>(g, method, src, dst, cfg, st);
    case DT_F16: return launch_m<__half>(g, method, src, dst, cfg, st);
    case DT_BF16: return launch_m<__nv_bfloat16>(g, method, src, dst, cfg, st);
    case DT_F32: return launch_m<float>(g, method, src, dst, cfg, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rs
