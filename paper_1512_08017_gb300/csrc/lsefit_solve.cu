// lsefit_solve.cu -- Gaussian elimination of the normal equations AX = B
// (Section II), one system per thread, FP64, partial pivoting, followed by
// the un-map of the coefficients.
#include "lsefit_device.cuh"
#include "lsefit_host.h"

namespace lsefit {

// One system per thread.  Systems of every degree up to NMAX share the
// padded elimination, so a warp never diverges on the degree.
template <int NMAX, bool CHOL>
__global__ void solve_kernel(const double* sums, int64_t count, int m_sums, int m, double eps,
                             const double* map, double* X, double* Xt, int32_t* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* row = sums + i * (3 * m_sums + 2);
    double c = 0.0, s = 1.0;
    bool ok = true;
    if (map) {
        c = map[2 * i];
        s = map[2 * i + 1];
        ok = isfinite(c) && isfinite(s) && s != 0.0;
    }
    const int st = solve_hankel_rt<NMAX, CHOL>(m, row, row + 2 * m_sums + 1, c, s, ok, eps,
                                         Xt ? Xt + i * (m + 1) : nullptr, X + i * (m + 1), m + 1);
    if (status) status[i] = st;
}

}  // namespace lsefit

using namespace lsefit;

static int launch_solve(bool chol, const double* sums, int64_t count, int m_sums, int m, int accum,
                        const double* map, double* X, double* Xt, int32_t* status, lsefit_stream_t stream) {
    if (count < 0 || m < 1 || m > LSEFIT_MAX_DEGREE || m_sums < m || m_sums > LSEFIT_MAX_DEGREE)
        return LSEFIT_ERR_INVALID_ARG;
    if (accum < LSEFIT_ACCUM_NAIVE || accum > LSEFIT_ACCUM_F64) return LSEFIT_ERR_INVALID_ARG;
    if (count == 0) return LSEFIT_OK;
    if (sums == nullptr || X == nullptr) return LSEFIT_ERR_INVALID_ARG;
    const int threads = 64;
    const int64_t blocks = (count + threads - 1) / threads;
    if (blocks > 0x7fffffffll) return LSEFIT_ERR_INVALID_ARG;
    typedef void (*kern_t)(const double*, int64_t, int, int, double, const double*, double*, double*, int32_t*);
    kern_t k;
    if (chol) k = m <= 1 ? solve_kernel<1, true> : m == 2 ? solve_kernel<2, true> : m == 3 ? solve_kernel<3, true>
                : m <= 5 ? solve_kernel<5, true> : solve_kernel<8, true>;
    else k = m <= 1 ? solve_kernel<1, false> : m == 2 ? solve_kernel<2, false> : m == 3 ? solve_kernel<3, false>
             : m <= 5 ? solve_kernel<5, false> : solve_kernel<8, false>;
    k<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(sums, count, m_sums, m, singular_eps(accum), map,
                                                              X, Xt, status);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}

extern "C" int lsefit_solve(const double* sums, int64_t count, int m_sums, int m, int accum,
                            const double* map, double* X, double* Xt, int32_t* status,
                            lsefit_stream_t stream) {
    return launch_solve(false, sums, count, m_sums, m, accum, map, X, Xt, status, stream);
}

extern "C" int lsefit_solve_cholesky(const double* sums, int64_t count, int m_sums, int m, int accum,
                                     const double* map, double* X, double* Xt, int32_t* status,
                                     lsefit_stream_t stream) {
    return launch_solve(true, sums, count, m_sums, m, accum, map, X, Xt, status, stream);
}

// ---------------------------------------------------------------------------
// Diagnostic: the eliminations' reciprocal on a caller's values (for tests).
// ---------------------------------------------------------------------------
namespace lsefit {
__global__ void reciprocal_kernel(const double* a, double* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = recip_f64(a[i]);
}
}  // namespace lsefit

extern "C" int lsefit_check_reciprocal(const double* a, double* out, int64_t n, lsefit_stream_t stream) {
    if (n < 0 || (n > 0 && (a == nullptr || out == nullptr))) return LSEFIT_ERR_INVALID_ARG;
    if (n == 0) return LSEFIT_OK;
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 0x7fffffffll) return LSEFIT_ERR_INVALID_ARG;
    reciprocal_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(a, out, n);
    return cudaGetLastError() == cudaSuccess ? LSEFIT_OK : LSEFIT_ERR_CUDA;
}
