// Kernels of the generalised fit, kind: weighted.
#include "lsefit_general.cuh"

namespace lsefit {
gen_kernel_t gen_pick_weighted(int m, int dtype, int accum) { return gen_pick<true, false>(m, dtype, accum); }
}  // namespace lsefit
