// Batched kernel instantiation: bf16 storage, f64 accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_bf16_f64, LSEFIT_BF16, LSEFIT_ACCUM_F64)
}  // namespace lsefit
