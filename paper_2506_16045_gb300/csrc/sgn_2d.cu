// 2d (doubly periodic) kernels.
#include "sgn_2d.h"

namespace sgn {

cudaError_t layout2d_create(Layout2d& L, const sgn_grid& g) {
  (void)L; (void)g;
  return cudaErrorNotSupported;
}
void layout2d_destroy(Layout2d& L) { cudaFree(L.work); L.work = nullptr; }
size_t layout2d_res_bytes(const Layout2d& L) { return 16 * (size_t)(L.P > 0 ? L.P : 1); }
cudaError_t launch_grad2d(const Layout2d&, const void*, const double*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_coeffs2d(const Layout2d&, const double*, const double*, int, SolveRec*,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_apply_G2d(const Layout2d&, const void*, const double*, const double*,
                             const double*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_precond2d(const Layout2d&, const void*, const SolveRec*, const double*, double*,
                             cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_pcg2d(const Layout2d&, const void*, const void*, int, const double*,
                         const double*, const double*, double*, const SolveRec*, int, double,
                         double, int, int, SolveRec*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_rhs2d(const Layout2d&, const void*, double, const double*, const double*,
                         const double*, const double*, double*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_lincomb2d(const Layout2d&, const double*, double*, const double* const*,
                             const double*, int, const double* const*, const double*, int, int,
                             cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_linimp_res2d(const Layout2d&, const void*, const SolveRec*, const double*,
                                const double*, const double*, const double*, void*,
                                cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_linimp_solve2d(const Layout2d&, const void*, const SolveRec*, const void*,
                                  const void*, double, double, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace sgn
