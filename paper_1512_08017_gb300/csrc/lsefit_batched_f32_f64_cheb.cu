// Batched kernel instantiation: f32 storage, f64 accumulation, Chebyshev basis.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE_CHEB(batched_f32_f64_cheb, LSEFIT_F32, LSEFIT_ACCUM_F64)
}  // namespace lsefit
