// Launch attributes kept per device and shared by every host thread.
//
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current
// device's context only, and a process may drive several devices from several
// threads (the server's worker thread beside the caller's), so the record of
// what was set, and the occupancy derived from it, is keyed by (device,
// kernel) under one mutex instead of a per-process static.
#include <map>
#include <mutex>
#include <tuple>

#include "gfbp_internal.cuh"

namespace gfbp {

namespace {

std::mutex g_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_set;                 // largest size enabled
std::map<std::tuple<int, const void*, int, size_t>, int> g_occupancy;     // CTAs per SM
std::map<int, int> g_sms, g_optin;

}  // namespace

cudaError_t kernel_prepare(const void* fn, int threads, size_t smem, int* occ) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (smem > 0) {
        // (the limit covers static and dynamic shared memory together, so it is
        // raised for any dynamic size above what was enabled before)
        size_t& set = g_smem_set[{dev, fn}];
        if (smem > set) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set = smem;
        }
    }
    const auto key = std::make_tuple(dev, fn, threads, smem);
    auto it = g_occupancy.find(key);
    if (it == g_occupancy.end()) {
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, threads, smem);
        if (e != cudaSuccess) return e;
        it = g_occupancy.emplace(key, o).first;
    }
    if (occ) *occ = it->second;
    return cudaSuccess;
}

static int device_attr(std::map<int, int>& cache, cudaDeviceAttr attr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache.find(dev);
    if (it == cache.end()) {
        int v = 0;
        cudaDeviceGetAttribute(&v, attr, dev);
        it = cache.emplace(dev, v).first;
    }
    return it->second;
}

int device_sms() {
    const int v = device_attr(g_sms, cudaDevAttrMultiProcessorCount);
    return v > 0 ? v : 1;
}

int device_optin_smem() { return device_attr(g_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin); }

}  // namespace gfbp
