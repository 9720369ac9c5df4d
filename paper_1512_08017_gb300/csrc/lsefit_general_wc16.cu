// Kernels of the generalised fit, Chebyshev basis with weights, degrees 9..16.
#include "lsefit_general.cuh"

namespace lsefit {
gen_kernel_t gen_pick_weighted_chebyshev_high(int m, int dtype, int accum) { return gen_pick_high<true>(m, dtype, accum); }
}  // namespace lsefit
