// 1d solve kernels for n = 2^14 (sgn_1d_pcg.cuh): two-CTA clusters of the n = 2^13 kernel,
// a translation unit of its own so the large instantiations compile in parallel.
#include "sgn_1d_pcg.cuh"

namespace sgn {
template cudaError_t pcg1d_launch<14, 2>(const PcgArgs&, int, int, cudaStream_t);
}  // namespace sgn
