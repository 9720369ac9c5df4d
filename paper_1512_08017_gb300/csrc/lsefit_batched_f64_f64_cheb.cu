// Batched kernel instantiation: f64 storage, f64 accumulation, Chebyshev basis.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE_CHEB(batched_f64_f64_cheb, LSEFIT_F64, LSEFIT_ACCUM_F64)
}  // namespace lsefit
