// Internal interface of the 2d (doubly periodic) kernels.
#pragma once
#include <cuda_runtime.h>

#include "sgn_internal.h"

namespace sgn {

struct Scal2d;   // device-resident scalars of one 2d solve (sgn_2d.cu)

// One 2d instance: fields [ny][nx] row-major; vector fields are two planes of P = nx ny.
// Spectra are half spectra [ny][H], H = nx/2 + 1; every half-plane buffer has 16 bytes
// per element so that it can hold complex float, double-float or double.
struct Layout2d {
  int nx = 0, ny = 0, lx = 0, ly = 0;
  double Lx = 0.0, Ly = 0.0;
  long long P = 0;          // points
  int H = 0;                // half width
  long long HP = 0;         // half-plane elements
  void* vec = nullptr;      // 14 half planes: b^ (0,1), x^ (2,3), r^ (4,5), p^ (6,7), d^ (8,9),
                            // G p / residual (10,11), spare (12,13)
  void* tp = nullptr;       // 4 transform half planes
  float* coef = nullptr;    // 6 coefficient planes (float parts)
  float* coef_lo = nullptr; // 6 coefficient planes (double-float remainders)
  double* parts = nullptr;  // per-block partial sums
  Scal2d* sc = nullptr;
  double* rhs_w = nullptr;  // 32 real planes of right-hand-side intermediates
  // Device-driven solves: one instantiated graph per [mixed][given coefficients], built on
  // first use, and the buffers its kernels address: staged eta [P], grad h [2P], b [2P],
  // x [2P], and two solve records (given coefficients in, report out).
  mutable cudaGraphExec_t solve_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  mutable bool solve_graph_off = false;   // building one failed: host-driven solves
  double* stage = nullptr;
  SolveRec* stage_rec = nullptr;
};

cudaError_t layout2d_create(Layout2d& L, const sgn_grid& g);
void layout2d_destroy(Layout2d& L);
size_t layout2d_res_bytes(const Layout2d& L);

cudaError_t launch_grad2d(const Layout2d& L, const void* tw64, const double* f, double* gradf,
                          cudaStream_t s);
cudaError_t launch_coeffs2d(const Layout2d& L, const double* eta, const double* gradh, int kind,
                            SolveRec* rec, cudaStream_t s);
cudaError_t launch_apply_G2d(const Layout2d& L, const void* tw64, const double* eta,
                             const double* gradh, const double* u, double* Gu, cudaStream_t s);
// Orszag's 2/3 rule (modes |jx| > nx/3 or |jy| > ny/3 set to zero) on eta - h, U and, if
// non-null, u (float64; uses the workspace planes)
cudaError_t launch_dealias2d(const Layout2d& L, const void* tw64, const double* h, double* eta,
                             double* U, double* u, cudaStream_t s);
// Non-constraint form in 2d (Eq:MomEq): f_eta = -div(eta u) and M (2 planes), float64;
// uses the right-hand-side planes of the layout
cudaError_t launch_rhs_nc2d(const Layout2d& L, const void* tw64, double g, const double* eta,
                            const double* u, const double* h, const double* gradh, double* f_eta,
                            double* M, cudaStream_t s);
cudaError_t launch_precond2d(const Layout2d& L, const void* tw64, const SolveRec* rec,
                             const double* r, double* z, cudaStream_t s);
// Runs as one cached graph whose refinement and inner loops are conditional (while) nodes
// driven by device-side decisions: no host round trip.  A stream under capture, or a graph
// the driver refuses, takes the host-driven path, which reads the stop flags back.
cudaError_t launch_pcg2d(const Layout2d& L, const void* tw64, const void* tw32, int precision,
                         const double* eta, const double* gradh, const double* b, double* x,
                         const SolveRec* given, int kind, double rtol, double rtol_inner,
                         int maxit, int max_refine, SolveRec* rec, cudaStream_t s);
// precision SGN_PREC_MIXED: transforms in double-float (pointwise work stays float64)
cudaError_t launch_rhs2d(const Layout2d& L, const void* tw64, const void* tw32, int precision,
                         double g, const double* eta, const double* u, const double* h,
                         const double* gradh, double* f_eta, double* f_U, cudaStream_t s);
cudaError_t launch_lincomb2d(const Layout2d& L, const double* dt, double* out,
                             const double* const* x, const double* a, int nx,
                             const double* const* f, const double* c, int nf, int components,
                             cudaStream_t s);
cudaError_t launch_linimp_res2d(const Layout2d& L, const void* tw64, const SolveRec* A,
                                const double* eta, const double* gradh, const double* u,
                                const double* U, void* res_hat, cudaStream_t s);
cudaError_t launch_linimp_solve2d(const Layout2d& L, const void* tw64, const SolveRec* A,
                                  const void* res1_hat, const void* res0_hat, double c1,
                                  double c0, double* u, cudaStream_t s);

}  // namespace sgn
