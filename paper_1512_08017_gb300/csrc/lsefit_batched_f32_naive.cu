// Batched kernel instantiation: f32 storage, naive accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_f32_naive, LSEFIT_F32, LSEFIT_ACCUM_NAIVE)
}  // namespace lsefit
