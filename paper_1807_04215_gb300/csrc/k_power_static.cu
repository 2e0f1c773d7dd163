// Shell power estimator with library-owned scratch (no allocation by anyone).
//
// gridspt_power needs a caller-allocated scratch buffer for its per-block
// partial sums. Some callers cannot allocate device memory at the point where
// they want a power spectrum: a host framework whose caching allocator already
// owns (nearly) all device memory and forbids foreign cudaMalloc calls, a
// plugin that is handed only input and output buffers, or code running with a
// fixed device-memory budget. For them this file holds the scratch in a
// file-scope __device__ array that is part of the library image: every GPU
// that loads libgridspt.so keeps these bytes until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) and cached; the first call on each device does this set-up.
#include <mutex>

#include "gridspt_internal.h"

namespace gridspt {

namespace {

constexpr int kMaxDevices = 64;

// kPowerMaxBlocks (1216) blocks x 2 sums x 64 bins x 8 bytes = 1,245,184 bytes per device.
static __device__ __align__(256) double g_power_scratch[(size_t)kPowerMaxBlocks * 2 * kMaxBins];
static_assert(sizeof(g_power_scratch) == (size_t)1245184, "static scratch size stated in gridspt.h");

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

}  // namespace

size_t power_static_scratch_bytes() { return sizeof(g_power_scratch); }

cudaError_t power_static_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_power_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool power_static_fits(const Geo& g, int nbins) {
    return (size_t)power_blocks(g) * 2 * nbins * sizeof(double) <= sizeof(g_power_scratch);
}

}  // namespace gridspt
