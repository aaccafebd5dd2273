// 1d solve and right-hand-side kernels for n = 2^6 .. 2^8 (sgn_1d_pcg.cuh, sgn_1d_rhs.cuh).
#include "sgn_1d_pcg.cuh"
#include "sgn_1d_rhs.cuh"

namespace sgn {
template cudaError_t pcg1d_launch<6, 1>(const PcgArgs&, int, int, cudaStream_t);
template cudaError_t pcg1d_launch<7, 1>(const PcgArgs&, int, int, cudaStream_t);
template cudaError_t pcg1d_launch<8, 1>(const PcgArgs&, int, int, cudaStream_t);
template cudaError_t rhs1d_launch<6, 1>(const RhsArgs&, int, int, cudaStream_t);
template cudaError_t rhs1d_launch<7, 1>(const RhsArgs&, int, int, cudaStream_t);
template cudaError_t rhs1d_launch<8, 1>(const RhsArgs&, int, int, cudaStream_t);
}  // namespace sgn
