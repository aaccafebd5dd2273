// 1d right-hand-side kernels for n = 2^12 on two-CTA clusters (sgn_1d_rhs.cuh), a form the
// layout can select per size class; a translation unit of its own so the instantiations
// compile in parallel.
#include "sgn_1d_rhs.cuh"

namespace sgn {
template cudaError_t rhs1d_launch<12, 2>(const RhsArgs&, int, int, cudaStream_t);
}  // namespace sgn
