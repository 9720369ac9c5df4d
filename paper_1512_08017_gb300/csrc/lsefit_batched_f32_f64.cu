// Batched kernel instantiation: f32 storage, f64 accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_f32_f64, LSEFIT_F32, LSEFIT_ACCUM_F64)
}  // namespace lsefit
