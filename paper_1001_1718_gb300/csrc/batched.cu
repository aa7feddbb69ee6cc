// Ragged batch: many images of uneven sizes, each with its own scale,
// channel count and method, resampled by one persistent kernel launch.
//
// The host cuts every image into output tiles (tile_w elements x tile_h
// rows, tile_h chosen per image so the staged footprint fits the block's
// shared memory), lays the images' tile counts out as an exclusive prefix
// sum, and uploads the descriptors and the prefix into the caller's
// workspace. The kernel runs one block per resident slot (SM count x blocks
// per SM); block b takes tiles b, b + gridDim.x, ..., finds each tile's image
// by binary search in the prefix and runs the same tile_body as the
// single-image kernel. No block waits on another.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <map>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "tile_body.cuh"

namespace rs {

struct BatchImage {
    const void* src;
    void* dst;
    int64_t src_pitch, dst_pitch;
    int H, W, Ho, Wo;
    int C, method, tiles_x, pad;
    int tile_w, tile_h, sh_max, swe_max;
};

template <int KT, typename T>
__device__ __forceinline__ void batch_tile_c(const Geom& g, const BatchImage& im, const TileCfg& cfg, int bx,
                                             int by, float* sm, unsigned int* fault)
{
    const T* s = static_cast<const T*>(im.src);
    T* d = static_cast<T*>(im.dst);
    switch (im.C) {
    case 1: tile_body<KT, 1, T>(g, s, d, cfg, bx, by, sm, fault); break;
    case 2: tile_body<KT, 2, T>(g, s, d, cfg, bx, by, sm, fault); break;
    case 3: tile_body<KT, 3, T>(g, s, d, cfg, bx, by, sm, fault); break;
    default: tile_body<KT, 4, T>(g, s, d, cfg, bx, by, sm, fault); break;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_batched(const BatchImage* __restrict__ imgs, const int64_t* __restrict__ start, int n, int64_t total,
          int coord, float a, unsigned int* fault)
{
    extern __shared__ __align__(16) float sm[];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        // image k with start[k] <= t < start[k + 1]
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
        }
        const BatchImage im = imgs[lo];
        const int64_t local = t - __ldg(start + lo);
        const int64_t count = __ldg(start + lo + 1) - __ldg(start + lo);
        if (local < 0 || local >= count) {   // uniform over the block
            if (threadIdx.x == 0) report_fault(fault, FAULT_BATCH_INDEX);
            continue;
        }
        Geom g;
        g.H = im.H; g.W = im.W; g.Ho = im.Ho; g.Wo = im.Wo; g.C = im.C;
        g.src_pitch = im.src_pitch;
        g.dst_pitch = im.dst_pitch;
        g.sp = PlaneMap{0, 0, 1};
        g.dp = PlaneMap{0, 0, 1};
        g.planes = 1;
        g.coord = coord;
        g.a = a;
        TileCfg cfg;
        cfg.tile_w = im.tile_w;
        cfg.tile_h = im.tile_h;
        cfg.threads = blockDim.x;
        cfg.sh_max = im.sh_max;
        cfg.swe_max = im.swe_max;
        cfg.smem = 0;
        const int bx = (int)(local % im.tiles_x), by = (int)(local / im.tiles_x);
        switch (im.method) {
        case M_NEAREST: batch_tile_c<1, T>(g, im, cfg, bx, by, sm, fault); break;
        case M_BILINEAR: batch_tile_c<2, T>(g, im, cfg, bx, by, sm, fault); break;
        default: batch_tile_c<4, T>(g, im, cfg, bx, by, sm, fault); break;
        }
        __syncthreads();   // the next tile reuses shared memory
    }
}

// ---------------------------------------------------------------------------
// Host side

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct BatchPlanHost {
    std::vector<BatchImage> imgs;
    std::vector<int64_t> start;
    size_t smem = 0;
    int threads = 256;
    size_t ws_bytes = 0;
    size_t off_start = 0;
};

static bool dim_ok(int v) { return v >= 1 && v <= 65535; }

// Tile shape of one image: tile_w elements, the tallest tile_h <= h_cap that
// fits `budget` bytes of shared memory, else the tallest that fits at all.
static bool image_tile(const Geom& g, int method, int tile_w, int h_cap, int threads, size_t budget, TileCfg& out)
{
    for (int pass = 0; pass < 2; ++pass) {
        for (int th = h_cap; th >= 1; th >>= 1) {
            TileCfg c{tile_w, th, threads, 0, 0, 0};
            if (!tiled_config(g, method, c)) continue;
            if (pass == 0 && c.smem > budget) continue;
            out = c;
            return true;
        }
    }
    return false;
}

static rs_status batch_prepare(const rs_image_desc* d, int n, int dtype, const rs_options& o, BatchPlanHost& P)
{
    if (!d || n < 1 || n > (1 << 20)) return RS_ERR_INVALID_ARG;
    if (dtype < RS_U8 || dtype > RS_F32) return RS_ERR_INVALID_ARG;
    rs_status s = check_options(o, RS_BILINEAR);
    if (s != RS_OK) return s;
    const int tile_w = o.tile_w ? o.tile_w : 512;
    const int h_cap = o.tile_h ? o.tile_h : 32;
    P.threads = o.threads ? o.threads : 256;
    if (P.threads != 128 && P.threads != 256) return RS_ERR_INVALID_ARG;
    const size_t es = dtype_size(dtype);
    std::vector<std::pair<const char*, int64_t>> srcs(n), dsts(n);
    P.imgs.resize(n);
    P.start.assign(n + 1, 0);
    P.smem = 0;
    for (int k = 0; k < n; ++k) {
        const rs_image_desc& x = d[k];
        if (!x.src || !x.dst) return RS_ERR_INVALID_ARG;
        if (!dim_ok(x.H) || !dim_ok(x.W) || !dim_ok(x.Ho) || !dim_ok(x.Wo)) return RS_ERR_INVALID_ARG;
        if (x.C < 1 || x.C > 4) return RS_ERR_INVALID_ARG;
        if (x.method < RS_NEAREST || x.method > RS_BICUBIC) return RS_ERR_INVALID_ARG;
        if (x.src_pitch < (int64_t)x.W * x.C || x.dst_pitch < (int64_t)x.Wo * x.C) return RS_ERR_INVALID_ARG;
        if (reinterpret_cast<uintptr_t>(x.src) % es || reinterpret_cast<uintptr_t>(x.dst) % es)
            return RS_ERR_ALIGNMENT;
        srcs[k] = {static_cast<const char*>(x.src), ((int64_t)(x.H - 1) * x.src_pitch + (int64_t)x.W * x.C) * (int64_t)es};
        dsts[k] = {static_cast<const char*>(x.dst), ((int64_t)(x.Ho - 1) * x.dst_pitch + (int64_t)x.Wo * x.C) * (int64_t)es};
        Geom g;
        g.H = x.H; g.W = x.W; g.Ho = x.Ho; g.Wo = x.Wo; g.C = x.C;
        g.src_pitch = x.src_pitch; g.dst_pitch = x.dst_pitch;
        g.sp = PlaneMap{0, 0, 1}; g.dp = PlaneMap{0, 0, 1};
        g.planes = 1; g.coord = o.coord; g.a = o.cubic_a;
        TileCfg c;
        if (!image_tile(g, x.method, tile_w, h_cap, P.threads, 72 * 1024, c)) return RS_ERR_UNSUPPORTED;
        BatchImage& im = P.imgs[k];
        std::memset(&im, 0, sizeof im);
        im.src = x.src; im.dst = x.dst;
        im.src_pitch = x.src_pitch; im.dst_pitch = x.dst_pitch;
        im.H = x.H; im.W = x.W; im.Ho = x.Ho; im.Wo = x.Wo; im.C = x.C; im.method = x.method;
        im.tile_w = c.tile_w; im.tile_h = c.tile_h; im.sh_max = c.sh_max; im.swe_max = c.swe_max;
        im.tiles_x = (int)(((int64_t)x.Wo * x.C + c.tile_w - 1) / c.tile_w);
        const int64_t tiles = (int64_t)im.tiles_x * ((x.Ho + c.tile_h - 1) / c.tile_h);
        P.start[k + 1] = P.start[k] + tiles;
        P.smem = std::max(P.smem, c.smem);
    }
    // No destination may overlap any source or another destination.
    for (int k = 0; k < n; ++k) {
        for (int l = 0; l < n; ++l) {
            if (overlaps(dsts[k].first, dsts[k].second, srcs[l].first, srcs[l].second)) return RS_ERR_INVALID_ARG;
            if (l != k && overlaps(dsts[k].first, dsts[k].second, dsts[l].first, dsts[l].second))
                return RS_ERR_INVALID_ARG;
        }
    }
    P.off_start = align256(sizeof(BatchImage) * (size_t)n);
    P.ws_bytes = P.off_start + sizeof(int64_t) * (size_t)(n + 1);
    return RS_OK;
}

template <typename T>
static void* batched_func() { return reinterpret_cast<void*>(&k_batched<T>); }

static void* batched_kernel(int dtype)
{
    switch (dtype) {
    case DT_U8: return batched_func<uint8_t>();
    case DT_F16: return batched_func<__half>();
    case DT_BF16: return batched_func<__nv_bfloat16>();
    default: return batched_func<float>();
    }
}

struct BatchLaunch {
    void* func;
    dim3 grid, block;
    size_t smem;
    const BatchImage* imgs;
    const int64_t* start;
    int n;
    int64_t total;
    int coord;
    float a;
    unsigned int* fault;
};

static cudaError_t batch_launch_params(const BatchPlanHost& P, int dtype, const rs_options& o, void* ws,
                                       BatchLaunch& L)
{
    L.func = batched_kernel(dtype);
    cudaError_t e = cudaFuncSetAttribute(L.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L.func, P.threads, P.smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
    const int64_t total = P.start.back();
    const int64_t blocks = std::min<int64_t>(total, (int64_t)num_sms() * per_sm);
    L.grid = dim3((unsigned)std::max<int64_t>(1, blocks));
    L.block = dim3(P.threads);
    L.smem = P.smem;
    L.imgs = static_cast<const BatchImage*>(ws);
    L.start = reinterpret_cast<const int64_t*>(static_cast<char*>(ws) + P.off_start);
    L.n = (int)P.imgs.size();
    L.total = total;
    L.coord = o.coord;
    L.a = o.cubic_a;
    L.fault = fault_word();
    return cudaSuccess;
}

static cudaError_t upload(const BatchPlanHost& P, void* ws, cudaStream_t st)
{
    std::vector<char> blob(P.ws_bytes, 0);
    std::memcpy(blob.data(), P.imgs.data(), sizeof(BatchImage) * P.imgs.size());
    std::memcpy(blob.data() + P.off_start, P.start.data(), sizeof(int64_t) * P.start.size());
    cudaError_t e = cudaMemcpyAsync(ws, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    // The host blob dies with this function: wait for the copy to finish.
    return cudaStreamSynchronize(st);
}

static cudaError_t launch_now(BatchLaunch& L, cudaStream_t st)
{
    void* args[] = {&L.imgs, &L.start, &L.n, &L.total, &L.coord, &L.a, &L.fault};
    cudaError_t e = cudaLaunchKernel(L.func, L.grid, L.block, args, L.smem, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

static rs_status check_ws(const BatchPlanHost& P, void* ws, size_t bytes)
{
    if (!ws || bytes < P.ws_bytes) return RS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) % 256) return RS_ERR_ALIGNMENT;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// Batched resampling without any allocation.
//
// Some callers cannot obtain device memory for the workspace: code running
// under an allocator that owns all device memory (a framework's caching
// pool or a fixed memory budget), real-time serving paths that forbid any
// allocation after start-up because cudaMalloc can block or fail, and plugin
// hosts that only hand out their own input and output buffers. For them the
// work list lives in a fixed array of device memory that the library itself
// declares (file scope, `static __device__`), so no call allocates: every GPU
// that loads the library holds kNoAllocBytes of it until the process exits.
//
// In host code the array's name is only a host-side handle, not a device
// address; its device address is looked up per device with
// cudaGetSymbolAddress (on the first call made on that device, with that
// device current) and passed to the kernel like any other pointer.
static constexpr int kNoAllocMaxImages = 4096;
static constexpr size_t kNoAllocImgBytes = ((sizeof(BatchImage) * kNoAllocMaxImages + 255) / 256) * 256;
static constexpr size_t kNoAllocBytes = kNoAllocImgBytes + sizeof(int64_t) * (kNoAllocMaxImages + 1);
static __device__ __align__(256) unsigned char g_batch_scratch[kNoAllocBytes];

static constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;                               // guards everything below
static void* g_noalloc_dev[kNoAllocMaxDevices];               // device address per device
static BatchImage g_noalloc_imgs[kNoAllocMaxImages];           // host staging (no heap use)
static int64_t g_noalloc_start[kNoAllocMaxImages + 1];

// Same validation and tiling as batch_prepare, written into the fixed
// host staging arrays instead of vectors.
static rs_status noalloc_prepare(const rs_image_desc* d, int n, int dtype, const rs_options& o, size_t& smem,
                                 int& threads)
{
    if (!d || n < 1) return RS_ERR_INVALID_ARG;
    if (n > kNoAllocMaxImages) return RS_ERR_WORKSPACE;
    if (dtype < RS_U8 || dtype > RS_F32) return RS_ERR_INVALID_ARG;
    rs_status s = check_options(o, RS_BILINEAR);
    if (s != RS_OK) return s;
    const int tile_w = o.tile_w ? o.tile_w : 512;
    const int h_cap = o.tile_h ? o.tile_h : 32;
    threads = o.threads ? o.threads : 256;
    if (threads != 128 && threads != 256) return RS_ERR_INVALID_ARG;
    const int64_t es = (int64_t)dtype_size(dtype);
    auto src_bytes = [&](const rs_image_desc& x) { return ((int64_t)(x.H - 1) * x.src_pitch + (int64_t)x.W * x.C) * es; };
    auto dst_bytes = [&](const rs_image_desc& x) { return ((int64_t)(x.Ho - 1) * x.dst_pitch + (int64_t)x.Wo * x.C) * es; };
    g_noalloc_start[0] = 0;
    smem = 0;
    for (int k = 0; k < n; ++k) {
        const rs_image_desc& x = d[k];
        if (!x.src || !x.dst) return RS_ERR_INVALID_ARG;
        if (!dim_ok(x.H) || !dim_ok(x.W) || !dim_ok(x.Ho) || !dim_ok(x.Wo)) return RS_ERR_INVALID_ARG;
        if (x.C < 1 || x.C > 4) return RS_ERR_INVALID_ARG;
        if (x.method < RS_NEAREST || x.method > RS_BICUBIC) return RS_ERR_INVALID_ARG;
        if (x.src_pitch < (int64_t)x.W * x.C || x.dst_pitch < (int64_t)x.Wo * x.C) return RS_ERR_INVALID_ARG;
        if (reinterpret_cast<uintptr_t>(x.src) % es || reinterpret_cast<uintptr_t>(x.dst) % es)
            return RS_ERR_ALIGNMENT;
        Geom g;
        g.H = x.H; g.W = x.W; g.Ho = x.Ho; g.Wo = x.Wo; g.C = x.C;
        g.src_pitch = x.src_pitch; g.dst_pitch = x.dst_pitch;
        g.sp = PlaneMap{0, 0, 1}; g.dp = PlaneMap{0, 0, 1};
        g.planes = 1; g.coord = o.coord; g.a = o.cubic_a;
        TileCfg c;
        if (!image_tile(g, x.method, tile_w, h_cap, threads, 72 * 1024, c)) return RS_ERR_UNSUPPORTED;
        BatchImage& im = g_noalloc_imgs[k];
        std::memset(&im, 0, sizeof im);
        im.src = x.src; im.dst = x.dst;
        im.src_pitch = x.src_pitch; im.dst_pitch = x.dst_pitch;
        im.H = x.H; im.W = x.W; im.Ho = x.Ho; im.Wo = x.Wo; im.C = x.C; im.method = x.method;
        im.tile_w = c.tile_w; im.tile_h = c.tile_h; im.sh_max = c.sh_max; im.swe_max = c.swe_max;
        im.tiles_x = (int)(((int64_t)x.Wo * x.C + c.tile_w - 1) / c.tile_w);
        g_noalloc_start[k + 1] = g_noalloc_start[k] + (int64_t)im.tiles_x * ((x.Ho + c.tile_h - 1) / c.tile_h);
        smem = std::max(smem, c.smem);
    }
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            if (overlaps(d[k].dst, dst_bytes(d[k]), d[l].src, src_bytes(d[l]))) return RS_ERR_INVALID_ARG;
            if (l != k && overlaps(d[k].dst, dst_bytes(d[k]), d[l].dst, dst_bytes(d[l]))) return RS_ERR_INVALID_ARG;
        }
    return RS_OK;
}

}  // namespace rs

extern "C" rs_status rs_resize_batched_noalloc(const rs_image_desc* d, int n, rs_dtype dtype, const rs_options* opt,
                                               void* stream)
{
    using namespace rs;
    const rs_options o = options_or_default(opt);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    size_t smem = 0;
    int threads = 256;
    rs_status s = noalloc_prepare(d, n, dtype, o, smem, threads);
    if (s != RS_OK) return s;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RS_ERR_UNSUPPORTED;
    if (!g_noalloc_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_noalloc_dev[dev] = p;
    }
    char* scratch = static_cast<char*>(g_noalloc_dev[dev]);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Pageable source: each copy returns once the host data has been staged,
    // so the staging arrays may be refilled by the next call.
    e = cudaMemcpyAsync(scratch, g_noalloc_imgs, sizeof(BatchImage) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kNoAllocImgBytes, g_noalloc_start, sizeof(int64_t) * (size_t)(n + 1),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    void* func = batched_kernel(dtype);
    if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_status(e);
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem)) != cudaSuccess)
        return cuda_status(e);
    const int64_t total = g_noalloc_start[n];
    const int64_t blocks = std::min<int64_t>(total, (int64_t)num_sms() * std::max(1, per_sm));
    const BatchImage* imgs = reinterpret_cast<const BatchImage*>(scratch);
    const int64_t* start = reinterpret_cast<const int64_t*>(scratch + kNoAllocImgBytes);
    int nn = n, coord = o.coord;
    float a = o.cubic_a;
    int64_t tot = total;
    unsigned int* fw = fault_word();
    void* args[] = {&imgs, &start, &nn, &tot, &coord, &a, &fw};
    e = cudaLaunchKernel(func, dim3((unsigned)std::max<int64_t>(1, blocks)), dim3(threads), args, smem, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_status(e);
}

using namespace rs;

struct rs_batched_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

extern "C" {

rs_status rs_resize_batched_workspace(const rs_image_desc* d, int n, rs_dtype dtype, size_t* bytes)
{
    if (!bytes) return RS_ERR_INVALID_ARG;
    rs_options o;
    rs_options_init(&o);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    *bytes = P.ws_bytes;
    return RS_OK;
}

rs_status rs_resize_batched(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace, size_t workspace_bytes,
                            const rs_options* opt, void* stream)
{
    const rs_options o = options_or_default(opt);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    if ((s = check_ws(P, workspace, workspace_bytes)) != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(P, workspace, st);
    if (e != cudaSuccess) return cuda_status(e);
    BatchLaunch L;
    if ((e = batch_launch_params(P, dtype, o, workspace, L)) != cudaSuccess) return cuda_status(e);
    return cuda_status(launch_now(L, st));
}

rs_status rs_batched_plan_create(const rs_image_desc* d, int n, rs_dtype dtype, void* workspace,
                                 size_t workspace_bytes, const rs_options* opt, void* stream, rs_batched_plan** plan)
{
    if (!plan) return RS_ERR_INVALID_ARG;
    *plan = nullptr;
    const rs_options o = options_or_default(opt);
    BatchPlanHost P;
    rs_status s = batch_prepare(d, n, dtype, o, P);
    if (s != RS_OK) return s;
    if ((s = check_ws(P, workspace, workspace_bytes)) != RS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(P, workspace, st);
    if (e != cudaSuccess) return cuda_status(e);
    BatchLaunch L;
    if ((e = batch_launch_params(P, dtype, o, workspace, L)) != cudaSuccess) return cuda_status(e);

    rs_batched_plan* p = new rs_batched_plan();
    cudaGetDevice(&p->device);
    void* args[] = {&L.imgs, &L.start, &L.n, &L.total, &L.coord, &L.a, &L.fault};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = L.func;
    kp.gridDim = L.grid;
    kp.blockDim = L.block;
    kp.sharedMemBytes = (unsigned)L.smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    if ((e = cudaGraphCreate(&p->graph, 0)) == cudaSuccess &&
        (e = cudaGraphAddKernelNode(&node, p->graph, nullptr, 0, &kp)) == cudaSuccess)
        e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return cuda_status(e);
    }
    *plan = p;
    return RS_OK;
}

rs_status rs_batched_plan_launch(rs_batched_plan* plan, void* stream)
{
    if (!plan || !plan->exec) return RS_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
}

rs_status rs_batched_plan_destroy(rs_batched_plan* plan)
{
    if (!plan) return RS_ERR_INVALID_ARG;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return RS_OK;
}

}  // extern "C"
