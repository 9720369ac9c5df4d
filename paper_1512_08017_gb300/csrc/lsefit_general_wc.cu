// Kernels of the generalised fit, kind: weighted chebyshev.
#include "lsefit_general.cuh"

namespace lsefit {
gen_kernel_t gen_pick_weighted_chebyshev(int m, int dtype, int accum) { return gen_pick<true, true>(m, dtype, accum); }
}  // namespace lsefit
