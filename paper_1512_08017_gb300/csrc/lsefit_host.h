// lsefit_host.h -- host-side helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace lsefit {

// Largest grid of the single-series reduction (bounds its workspace).
constexpr int kMaxGrid = 4096;
// Alignment of workspace regions.
constexpr size_t kAlign = 256;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// SM count of the current device (cached per device).  Returns 0 on error.
int current_sm_count(int* device_out);

// Resident blocks per SM of `kernel` at `threads` threads and `smem` dynamic
// shared memory (cached per kernel).  Returns at least 1.
int occupancy_blocks(const void* kernel, int threads, size_t smem);

// Device address of a point array: device or managed memory as is; host
// memory only when registered with CUDA (pinned), through the address CUDA
// reports for it.  Unregistered host memory gives LSEFIT_ERR_INVALID_ARG.
int resolve_device_pointer(const void*& ptr);

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int elem_size(int dtype) { return dtype == 0 ? 8 : (dtype == 1 ? 4 : 2); }

// Launch of a kernel that may start before the kernel ahead of it on the
// stream has finished (programmatic dependent launch): the kernel must call
// griddep_wait() before it reads anything its predecessor writes.  Inside a
// CUDA graph capture the dependency becomes a programmatic graph edge.
template <typename... Params, typename... Args>
inline cudaError_t launch_after_prior(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                                      cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lsefit
