// 1d solve kernels for n = 2^12 on two-CTA clusters (sgn_1d_pcg.cuh), a form the layout can
// select per size class; a translation unit of its own so the instantiations compile in
// parallel.
#include "sgn_1d_pcg.cuh"

namespace sgn {
template cudaError_t pcg1d_launch<12, 2>(const PcgArgs&, int, int, cudaStream_t);
}  // namespace sgn
