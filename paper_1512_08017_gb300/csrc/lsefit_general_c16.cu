// Kernels of the generalised fit, Chebyshev basis, degrees 9..16.
#include "lsefit_general.cuh"

namespace lsefit {
gen_kernel_t gen_pick_chebyshev_high(int m, int dtype, int accum) { return gen_pick_high<false>(m, dtype, accum); }
}  // namespace lsefit
