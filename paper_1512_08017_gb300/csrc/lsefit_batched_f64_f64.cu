// Batched kernel instantiation: f64 storage, f64 accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_f64_f64, LSEFIT_F64, LSEFIT_ACCUM_F64)
}  // namespace lsefit
