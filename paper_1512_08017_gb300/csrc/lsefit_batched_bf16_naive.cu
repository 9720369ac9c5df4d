// Batched kernel instantiation: bf16 storage, naive accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_bf16_naive, LSEFIT_BF16, LSEFIT_ACCUM_NAIVE)
}  // namespace lsefit
