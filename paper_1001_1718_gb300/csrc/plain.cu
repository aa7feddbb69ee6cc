// Plain kernel: one thread per output pixel, every tap read from global
// memory, blocks of bw x bh threads mapped onto the output by Eq. 6
// (p_x = b_x * b_width + t_x, p_y = b_y * b_height + t_y; Sec. III.A).
// This is the paper's design (Sec. III) on this GPU and the comparison
// baseline for the tiled kernels; it computes the same FP32 arithmetic in
// the same order (horizontal taps first, then vertical).
#include "rs_common.cuh"

namespace rs {

template <int KT, typename T>
__global__ void k_plain(const Geom g, const T* __restrict__ src, T* __restrict__ dst)
{
    const int px = blockIdx.x * blockDim.x + threadIdx.x;   // Eq. 6
    const int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= g.Wo || py >= g.Ho) return;
    const int plane = blockIdx.z;
    const T* s = src + g.sp.offset(plane);
    T* d = dst + g.dp.offset(plane) + (int64_t)py * g.dst_pitch + (int64_t)px * g.C;

    float wx[KT], wy[KT];
    const int fx = taps<KT>(px, g.W, g.Wo, g.coord, g.a, wx);
    const int fy = taps<KT>(py, g.H, g.Ho, g.coord, g.a, wy);
    int ix[KT], iy[KT];
    #pragma unroll
    for (int q = 0; q < KT; ++q) {
        ix[q] = clampi(fx + q, g.W);
        iy[q] = clampi(fy + q, g.H);
    }
    for (int c = 0; c < g.C; ++c) {
        float v = 0.0f;
        #pragma unroll
        for (int p = 0; p < KT; ++p) {
            const T* row = s + (int64_t)iy[p] * g.src_pitch + c;
            float h = 0.0f;
            #pragma unroll
            for (int q = 0; q < KT; ++q) h = fmaf(wx[q], Store<T>::load(row + (int64_t)ix[q] * g.C), h);
            v = fmaf(wy[p], h, v);
        }
        Store<T>::put(d + c, v);
    }
}

template <int KT, typename T>
static cudaError_t launch_t(const Geom& g, const void* src, void* dst, int bw, int bh,
                            cudaStream_t st)
{
    dim3 block(bw, bh);
    dim3 grid((g.Wo + bw - 1) / bw, (g.Ho + bh - 1) / bh, g.planes);
    k_plain<KT, T><<<grid, block, 0, st>>>(g, static_cast<const T*>(src), static_cast<T*>(dst));
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_m(const Geom& g, int method, const void* src, void* dst, int bw, int bh,
                            cudaStream_t st)
{
    switch (method) {
    case M_NEAREST: return launch_t<1, T>(g, src, dst, bw, bh, st);
    case M_BILINEAR: return launch_t<2, T>(g, src, dst, bw, bh, st);
    case M_BICUBIC: return launch_t<4, T>(g, src, dst, bw, bh, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_plain(const Geom& g, int method, int dtype, const void* src, void* dst,
                         int bw, int bh, cudaStream_t st)
{
    switch (dtype) {
    case DT_U8: return launch_m<uint8_t>(g, method, src, dst, bw, bh, st);
    case DT_F16: return launch_m<__half>(g, method, src, dst, bw, bh, st);
    case DT_BF16: return launch_m<__nv_bfloat16>(g, method, src, dst, bw, bh, st);
    case DT_F32: return launch_m<float>(g, method, src, dst, bw, bh, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rs
