// 1d right-hand-side kernels for n = 2^14 (sgn_1d_rhs.cuh): two-CTA clusters of the n = 2^13
// kernel, a translation unit of its own so the large instantiations compile in parallel.
#include "sgn_1d_rhs.cuh"

namespace sgn {
template cudaError_t rhs1d_launch<14, 2>(const RhsArgs&, int, int, cudaStream_t);
}  // namespace sgn
