// Kernels of the generalised fit, kind: chebyshev.
#include "lsefit_general.cuh"

namespace lsefit {
gen_kernel_t gen_pick_chebyshev(int m, int dtype, int accum) { return gen_pick<false, true>(m, dtype, accum); }
}  // namespace lsefit
