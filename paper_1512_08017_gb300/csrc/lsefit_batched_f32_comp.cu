// Batched kernel instantiation: f32 storage, comp accumulation.
#include "lsefit_batched.cuh"

namespace lsefit {
LSEFIT_BATCHED_INSTANTIATE(batched_f32_comp, LSEFIT_F32, LSEFIT_ACCUM_COMP)
}  // namespace lsefit
