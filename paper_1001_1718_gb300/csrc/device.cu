// Per-device state of the library: the fault word and cached device limits.
// The fault word is a static __device__ variable; host code must not use its
// name as a device address, so its address is resolved per device with
// cudaGetSymbolAddress (with that device current) and passed to kernels.
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "rs_internal.h"

namespace rs {

static __device__ unsigned int g_fault_word;

static constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static unsigned int* g_fault_ptr[kMaxDevices];
static size_t g_smem[kMaxDevices];
static int g_sms[kMaxDevices];
static std::string g_tag[kMaxDevices];

static int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

unsigned int* fault_word()
{
    const int dev = current_device();
    if (dev < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_fault_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fault_word) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        g_fault_ptr[dev] = static_cast<unsigned int*>(p);
    }
    return g_fault_ptr[dev];
}

size_t max_smem_per_block()
{
    const int dev = current_device();
    if (dev < 0) return 48 * 1024;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_smem[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 48 * 1024;
        g_smem[dev] = (size_t)v;
    }
    return g_smem[dev];
}

// Dynamic shared-memory limits already raised, per (device, kernel), and
// resident blocks per SM, per (device, kernel, threads, bytes): each driver
// query runs once, not on every launch.
static std::map<std::pair<int, const void*>, size_t> g_smem_set;
static std::map<std::tuple<int, const void*, int, size_t>, int> g_occupancy;

cudaError_t prepare_kernel(const void* func, size_t smem, int threads, int* per_sm)
{
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    size_t& set = g_smem_set[{dev, func}];
    if (smem > set) {
        const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    if (per_sm) {
        const auto key = std::make_tuple(dev, func, threads, smem);
        auto it = g_occupancy.find(key);
        if (it == g_occupancy.end()) {
            int v = 0;
            const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, func, threads, smem);
            if (e != cudaSuccess) return e;
            if (g_occupancy.size() >= 4096) g_occupancy.clear();   // many shapes: start over
            it = g_occupancy.emplace(key, v).first;
        }
        *per_sm = it->second;
    }
    return cudaSuccess;
}

int num_sms()
{
    const int dev = current_device();
    if (dev < 0) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        g_sms[dev] = v;
    }
    return g_sms[dev];
}

// "<device name>/cc<major><minor>/cudart<version>" with spaces replaced, for
// tuning-cache keys: a cache from another GPU model or CUDA runtime does not
// match.
const std::string& device_tag()
{
    static const std::string none = "nodevice";
    const int dev = current_device();
    if (dev < 0) return none;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_tag[dev].empty()) {
        cudaDeviceProp prop;
        int rt = 0;
        std::string t;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
            t = prop.name;
            t += "/cc" + std::to_string(prop.major) + std::to_string(prop.minor);
        } else {
            (void)cudaGetLastError();
            t = "unknown";
        }
        if (cudaRuntimeGetVersion(&rt) == cudaSuccess) t += "/cudart" + std::to_string(rt);
        else (void)cudaGetLastError();
        for (char& ch : t)
            if (ch == ' ' || ch == ';' || ch == '\t') ch = '_';
        g_tag[dev] = t;
    }
    return g_tag[dev];
}

int method_taps(int method)
{
    return method == M_NEAREST ? 1 : method == M_BILINEAR ? 2 : 4;
}

size_t dtype_size(int dtype)
{
    return dtype == DT_U8 ? 1 : dtype == DT_F32 ? 4 : 2;
}

// Reads and clears the current device's fault word after synchronising `st`.
cudaError_t read_fault(cudaStream_t st, unsigned int* code)
{
    unsigned int* fw = fault_word();
    *code = 0;
    if (!fw) return cudaErrorInvalidSymbol;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(code, fw, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    return cudaMemcpy(fw, &zero, sizeof(unsigned int), cudaMemcpyHostToDevice);
}

}  // namespace rs
