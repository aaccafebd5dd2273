// 1d solve kernels for n = 2^11 (sgn_1d_pcg.cuh), a translation unit of its own so the
// large instantiations compile in parallel.
#include "sgn_1d_pcg.cuh"

namespace sgn {
template cudaError_t pcg1d_launch<11, 1>(const PcgArgs&, int, int, cudaStream_t);
}  // namespace sgn
