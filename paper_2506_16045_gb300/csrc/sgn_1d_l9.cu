// 1d solve and right-hand-side kernels for n = 2^9 (sgn_1d_pcg.cuh, sgn_1d_rhs.cuh), one
// translation unit per size so the instantiations compile in parallel.
#include "sgn_1d_pcg.cuh"
#include "sgn_1d_rhs.cuh"

namespace sgn {
template cudaError_t pcg1d_launch<9, 1>(const PcgArgs&, int, int, cudaStream_t);
template cudaError_t rhs1d_launch<9, 1>(const RhsArgs&, int, int, cudaStream_t);
}  // namespace sgn
