// lsefit_general.cu -- host side of the generalised single-series fit
// (per-point weights, Chebyshev basis): argument checks, launch shape and
// the C entry points.  The kernels are in lsefit_general.cuh, instantiated
// one kind per translation unit (lsefit_general_{w,c,wc}.cu).
#include <mutex>
#include <unordered_map>

#include "lsefit_general.cuh"
#include "lsefit_host.h"

using namespace lsefit;

// Threads per block a general kernel was compiled for (its __launch_bounds__),
// per device and kernel.
static int block_threads_of(const void* kernel) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return kGenBlock;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache[dev].find(kernel);
    if (it != cache[dev].end()) return it->second;
    cudaFuncAttributes a;
    int t = kGenBlock;
    if (cudaFuncGetAttributes(&a, kernel) == cudaSuccess && a.maxThreadsPerBlock >= 32) t = a.maxThreadsPerBlock;
    else (void)cudaGetLastError();
    cache[dev][kernel] = t;
    return t;
}

extern "C" size_t lsefit_fit_general_workspace_size(int m) {
    if (m < 1 || m > LSEFIT_MAX_DEGREE_CHEBYSHEV) return 0;
    const size_t fit_ws = m <= LSEFIT_MAX_DEGREE ? lsefit_powersums_workspace_size(m) : 0;
    const size_t gen_ws = kAlign + align_up((size_t)kMaxGrid * (3 * m + 2) * sizeof(double), kAlign);
    return gen_ws > fit_ws ? gen_ws : fit_ws;
}

extern "C" int lsefit_fit_general(const void* x, const void* y, const void* w, int64_t n, int dtype, int m,
                                  int m_lo, int accum, int basis, const double* interval, double* X, double* Xb,
                                  double* sums, double* map, int32_t* status, void* workspace,
                                  size_t workspace_bytes, lsefit_stream_t stream) {
    if (basis != LSEFIT_BASIS_MONOMIAL && basis != LSEFIT_BASIS_CHEBYSHEV) return LSEFIT_ERR_INVALID_ARG;
    const int mmax = basis == LSEFIT_BASIS_CHEBYSHEV ? LSEFIT_MAX_DEGREE_CHEBYSHEV : LSEFIT_MAX_DEGREE;
    if (m < 1 || m > mmax || n < 0 || m_lo < 1 || m_lo > m) return LSEFIT_ERR_INVALID_ARG;
    if (X == nullptr || status == nullptr) return LSEFIT_ERR_INVALID_ARG;
    if (dtype < LSEFIT_F64 || dtype > LSEFIT_BF16) return LSEFIT_ERR_INVALID_ARG;
    if (accum < LSEFIT_ACCUM_NAIVE || accum > LSEFIT_ACCUM_F64) return LSEFIT_ERR_INVALID_ARG;
    if (dtype == LSEFIT_F64 && accum != LSEFIT_ACCUM_F64) return LSEFIT_ERR_UNSUPPORTED;
    if (w == nullptr && basis == LSEFIT_BASIS_MONOMIAL)  // the paper's objective: the tuned pass
        return lsefit_fit(x, y, n, dtype, m, m_lo, accum, interval, X, Xb, sums, map, status, workspace,
                          workspace_bytes, stream);
    if (n > 0 && (x == nullptr || y == nullptr)) return LSEFIT_ERR_INVALID_ARG;
    if (n >= (int64_t(1) << 53)) return LSEFIT_ERR_INVALID_ARG;
    if (workspace == nullptr || !aligned(workspace, kAlign)) return LSEFIT_ERR_WORKSPACE;
    if (workspace_bytes < lsefit_fit_general_workspace_size(m)) return LSEFIT_ERR_WORKSPACE;
    if (n > 0) {
        if (resolve_device_pointer(x) != LSEFIT_OK || resolve_device_pointer(y) != LSEFIT_OK) return LSEFIT_ERR_INVALID_ARG;
        if (w != nullptr && resolve_device_pointer(w) != LSEFIT_OK) return LSEFIT_ERR_INVALID_ARG;
    }
    const bool cheb = basis == LSEFIT_BASIS_CHEBYSHEV;
    gen_kernel_t k;
    if (m > LSEFIT_MAX_DEGREE)  // Chebyshev only (checked above)
        k = w != nullptr ? gen_pick_weighted_chebyshev_high(m, dtype, accum) : gen_pick_chebyshev_high(m, dtype, accum);
    else
        k = w != nullptr ? (cheb ? gen_pick_weighted_chebyshev(m, dtype, accum) : gen_pick_weighted(m, dtype, accum))
                         : gen_pick_chebyshev(m, dtype, accum);
    if (k == nullptr) return LSEFIT_ERR_UNSUPPORTED;
    GenParams p;
    p.x = x;
    p.y = y;
    p.w = w;
    p.n = n;
    p.interval = interval;
    p.sums = sums;
    p.map_out = map;
    p.ticket = static_cast<unsigned int*>(workspace);
    p.partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + kAlign);
    p.m_lo = m_lo;
    p.eps = singular_eps(accum);
    p.X = X;
    p.Xb = Xb;
    p.status = status;
    int dev = 0;
    const int sms = current_sm_count(&dev);
    if (sms <= 0) return LSEFIT_ERR_CUDA;
    const int threads = block_threads_of(reinterpret_cast<const void*>(k));
    const int occ = occupancy_blocks(reinterpret_cast<const void*>(k), threads, 0);
    const int64_t work = (n + 16 / elem_size(dtype) - 1) / (16 / elem_size(dtype));
    int64_t grid = (int64_t)sms * occ;
    const int64_t want = (work + 2 * threads - 1) / (2 * threads);
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    if (grid > kMaxGrid) grid = kMaxGrid;
    k<<<(unsigned)grid, threads, 0, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}
