// Batched kernel instantiation: bf16 storage, comp accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_bf16_comp, LSEFIT_BF16, LSEFIT_ACCUM_COMP)
}  // namespace lsefit
