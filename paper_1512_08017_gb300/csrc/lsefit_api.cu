// lsefit_api.cu -- status strings, version, and the per-device caches of
// launch parameters used by every entry point.
#include <mutex>
#include <unordered_map>

#include "lsefit.h"
#include "lsefit_host.h"

namespace lsefit {

int current_sm_count(int* device_out) {
    static std::mutex mu;
    static int cache[256] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 0;
    if (device_out) *device_out = dev;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = sms;
    }
    return cache[dev];
}

int occupancy_blocks(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache[dev].find(kernel);
    if (it != cache[dev].end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1)
        nb = 1;
    cache[dev][kernel] = nb;
    return nb;
}

// Device address of a point array: device/managed memory as is; host memory
// only when it is registered with CUDA (pinned), through the address CUDA
// reports for it.  Unregistered host memory is rejected.
int resolve_device_pointer(const void*& ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return LSEFIT_ERR_INVALID_ARG;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return LSEFIT_OK;
    if (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr) {
        ptr = a.devicePointer;
        return LSEFIT_OK;
    }
    return LSEFIT_ERR_INVALID_ARG;
}

}  // namespace lsefit

extern "C" const char* lsefit_status_string(int code) {
    switch (code) {
        case LSEFIT_OK: return "ok";
        case LSEFIT_ERR_INVALID_ARG: return "invalid argument";
        case LSEFIT_ERR_N_TOO_SMALL: return "fewer than m+1 points";
        case LSEFIT_ERR_SINGULAR: return "singular normal matrix";
        case LSEFIT_ERR_NONFINITE: return "non-finite power sums";
        case LSEFIT_ERR_BAD_INTERVAL: return "bad interval";
        case LSEFIT_ERR_WORKSPACE: return "workspace too small or misaligned";
        case LSEFIT_ERR_CUDA: return "CUDA error";
        case LSEFIT_ERR_UNSUPPORTED: return "unsupported dtype/accumulation";
        case LSEFIT_ERR_SCRATCH_LIMIT: return "request exceeds the static scratch of lsefit_fit_noalloc";
        default: return "unknown status";
    }
}

extern "C" int lsefit_abi_version(void) { return LSEFIT_ABI_VERSION; }
