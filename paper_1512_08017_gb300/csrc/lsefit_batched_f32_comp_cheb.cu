// Batched kernel instantiation: f32 storage, comp accumulation, Chebyshev basis.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE_CHEB(batched_f32_comp_cheb, LSEFIT_F32, LSEFIT_ACCUM_COMP)
}  // namespace lsefit
