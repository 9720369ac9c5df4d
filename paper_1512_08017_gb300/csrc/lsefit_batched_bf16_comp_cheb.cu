// Batched kernel instantiation: bf16 storage, comp accumulation, Chebyshev basis.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE_CHEB(batched_bf16_comp_cheb, LSEFIT_BF16, LSEFIT_ACCUM_COMP)
}  // namespace lsefit
