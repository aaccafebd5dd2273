// 1d right-hand-side kernels for n = 2^11 (sgn_1d_rhs.cuh), a translation unit of its own so
// the large instantiations compile in parallel.
#include "sgn_1d_rhs.cuh"

namespace sgn {
template cudaError_t rhs1d_launch<11, 1>(const RhsArgs&, int, int, cudaStream_t);
}  // namespace sgn
