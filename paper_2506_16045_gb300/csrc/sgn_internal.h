// Internal (C++) interface between the C ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgn.h"

namespace sgn {

constexpr int kTwiddleLog2 = 14;                 // twiddle table resolution: n <= 16384 per axis
constexpr int kTwiddleN = 1 << kTwiddleLog2;
// The float32 twiddle allocation also holds the double-float table right after it:
// [ float32 table, kTw32Bytes ][ double-float table, kTwDfBytes ].
constexpr size_t kTw64Bytes = (size_t)16 * kTwiddleN;
constexpr size_t kTw32Bytes = (size_t)8 * kTwiddleN;
constexpr size_t kTwDfBytes = (size_t)16 * kTwiddleN;

// One 1d periodic instance inside a packed batch.  Real fields of instance i occupy
// [off, off + n) of every packed array; the spectral workspace of the instance starts at
// ws (in units of complex doubles) and holds kWsVectors half spectra of n/2 + 1 modes.
struct Inst1d {
  int n;
  int log2n;             // log2 n, or 0 for a size that is not a power of two
  double L;
  long long off;
  long long ws;
  long long tw;          // sizes that are not powers of two: first entry of the n's twiddles
  long long gbuf;        // and, above the shared-memory limit, their global transform
                         // buffers' offset (complex doubles; -1: shared memory)
};

// Preconditioner coefficients and solve report per instance (device resident).
struct SolveRec {
  double sigma, alpha, kappa_ub, eta_min, eta_max;
  double ratio;          // final sqrt(r.A^{-1}r)/sqrt(b.A^{-1}b) (FP64 residual in the mixed path)
  int flat;
  int iters;             // PCG iterations (inner iterations summed over refinements)
  int refinements;       // FP32 inner solves (mixed) or 0 (FP64)
  int status;            // sgn_status of this instance
};

constexpr int kWsVectors = 6;          // half-spectrum vectors per instance in the workspace
constexpr int kMaxLog1d = 14;          // 1d n <= 16384 (n = 16384: two-CTA clusters)
constexpr int kSmemLog1d = 13;         // largest 1d n whose float64 transform fits in one CTA
constexpr int kClusterLog1d = 12;      // smallest 1d log2 n with a two-CTA cluster form
constexpr int kGenericClass = 0;       // size class of the 1d n that are not powers of two
// The size classes in launch order: the largest power of two first, the generic class last.
constexpr int kNumClassSlots = kMaxLog1d - 3 + 2;
inline int class_at(int i) { return i <= kMaxLog1d - 3 ? kMaxLog1d - i : kGenericClass; }

struct Layout1d {
  int count = 0;
  long long points = 0;                // sum of n
  int maxn = 0;                        // largest n
  long long ws_cplx = 0;               // workspace size in complex doubles
  Inst1d* d_inst = nullptr;            // device copy
  Inst1d* h_inst = nullptr;            // host copy
  int* d_ids = nullptr;                // instance ids grouped by size class
  int class_begin[16] = {0};           // per log2n: [begin, end) into ids; class
  int class_end[16] = {0};             // kGenericClass: the sizes that are not powers of two
  // sizes n = 2^a 3^b 5^c that are not powers of two (the generic kernels): their twiddle
  // tables (float64, float32, double-float, mr_tw_len entries each) and the largest such n
  void* mr_tw = nullptr;
  long long mr_tw_len = 0;
  int mr_smem_n = 0;                   // largest such n with shared-memory buffers
  void* mr_big = nullptr;              // global transform buffers of the larger ones
  // float64 transform buffers (n complex doubles per instance) of the cta_fft kernels for
  // the instances above kSmemLog1d, indexed by position in their size class
  void* big = nullptr;
  // CTAs per instance of each size class's solve (form) and right-hand side (rform; 0: the
  // default, one CTA up to kSmemLog1d and two above, and the right-hand side as the solve);
  // set_form(s) / autotune change them for the classes from kClusterLog1d, and `gen` counts
  // the changes (captured step graphs hold the old forms)
  int form[16] = {0};
  int rform[16] = {0};                 // the right-hand side's own form (0: as the solve's)
  int gen = 0;
  int ctas(int l) const { return form[l] ? form[l] : (l > kSmemLog1d ? 2 : 1); }
  int rhs_ctas(int l) const { return rform[l] ? rform[l] : ctas(l); }
  // side streams and events for running size classes concurrently (null: one stream)
  cudaStream_t side[16] = {nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[16] = {nullptr};
};

// Launchers (all asynchronous on `stream`; return cudaError_t of the launch).
cudaError_t twiddles_init(void* tw64, void* tw32, cudaStream_t s);

cudaError_t launch_deriv1d(const Layout1d& lay, const void* tw64, const double* f, double* fx,
                           cudaStream_t s);
cudaError_t launch_apply_G1d(const Layout1d& lay, const void* tw64, const double* eta,
                             const double* hx, const double* u, double* Gu, cudaStream_t s);
cudaError_t launch_coeffs1d(const Layout1d& lay, const double* eta, const double* hx, int kind,
                            SolveRec* rec, cudaStream_t s);
cudaError_t launch_precond1d(const Layout1d& lay, const void* tw64, const SolveRec* rec,
                             const double* r, double* z, cudaStream_t s);
// precision: SGN_PREC_FP64 or SGN_PREC_MIXED.  `given` (nullable) holds preconditioner
// coefficients per instance; otherwise they are computed from eta and hx (kind).
cudaError_t launch_pcg1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         const double* eta, const double* hx, const double* b, double* x,
                         const SolveRec* given, int kind, double rtol, double rtol_inner,
                         int maxit, int max_refine, SolveRec* rec, void* ws, float* coef_df,
                         cudaStream_t s);
cudaError_t launch_rhs1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         double g, const double* eta,
                         const double* u, const double* h, const double* hx, double* f_eta,
                         double* f_U, double* scratch, cudaStream_t s);
// Solve and right-hand side of a time-stepping stage, passing u_x between them: the solve
// (as launch_pcg1d with computed coefficients of `kind`) also stores x_x in the first plane
// of `scratch` (double-float for MIXED, float64 otherwise), and the right-hand side (as
// launch_rhs1d at u = x) takes it from there: six transforms instead of eight.
cudaError_t launch_pcg1d_ux(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, const double* eta, const double* hx, const double* b,
                            double* x, int kind, double rtol, double rtol_inner, int maxit,
                            int max_refine, SolveRec* rec, void* ws, float* coef_df,
                            double* scratch, cudaStream_t s);
cudaError_t launch_rhs1d_ux(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, double g, const double* eta, const double* u,
                            const double* h, const double* hx, double* f_eta, double* f_U,
                            double* scratch, cudaStream_t s);
// out = base + sum_j c_j dt_i f_j over up to 4 terms (per-instance dt from `dt`)
cudaError_t launch_axpy1d(const Layout1d& lay, const double* dt, double* out, const double* base,
                          int nterms, const double* const* f, const double* c, double scale,
                          cudaStream_t s);
// Orszag's 2/3 rule on a new level: modes |j| > n/3 of eta - h, U and (non-null) u set to 0
// (transforms in float64, or double-float for SGN_PREC_MIXED)
cudaError_t launch_dealias1d(const Layout1d& lay, const void* tw64, const void* tw32,
                             int precision, const double* h, double* eta, double* U, double* u,
                             cudaStream_t s);
// Non-constraint form (Eq:dswe / Eq:MomEq): f_eta = -(eta u)_x and M, the u_t-free terms
// with G u_t = M (transforms in float64, or double-float for SGN_PREC_MIXED); scratch:
// 2 P doubles
cudaError_t launch_rhs_nc1d(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, double g, const double* eta, const double* u,
                            const double* h, const double* hx, double* f_eta, double* M,
                            double* scratch, cudaStream_t s);
// SBDF2 velocity update in one launch (transforms in float64, or double-float for
// SGN_PREC_MIXED): res1_hat = (sigma + alpha k^2) u_hat - (G u - U)_hat, and with `solve`
// u_out <- A^{-1} iFFT(c1 res1_hat + c0 res0_hat) (u_out null: u in place).  ux_out
// (nullable): u_x in the transforms' precision, as the solve's u_x hand-off stores it.
cudaError_t launch_linimp_step1d(const Layout1d& lay, const void* tw64, const void* tw32,
                                 int precision, const SolveRec* A, const double* eta,
                                 const double* hx, double* u, const double* U,
                                 const void* res0_hat, void* res1_hat, double c1, double c0,
                                 bool solve, void* ws, double* u_out, void* ux_out,
                                 cudaStream_t s);

// Sizes n = 2^a 3^b 5^c (a >= 1) that are not powers of two, 6 <= n <= 16384: one CTA per
// instance with a mixed-radix transform in shared memory (n <= 6144; above, in global
// memory) (sgn_1d_mr.cu).  Each launches the generic instances ids[first, first + num) of
// the layout.
bool mr_size_ok(int n);
bool mr_in_smem(int n);
long long mr_twiddle_len(int n);
cudaError_t mr_twiddles_init(int n, long long off, const Layout1d& lay, cudaStream_t s);
cudaError_t mr_launch_deriv(const Layout1d& lay, int first, int num, const double* f,
                            double* fx, cudaStream_t s);
cudaError_t mr_launch_apply_G(const Layout1d& lay, int first, int num, const double* eta,
                              const double* hx, const double* u, double* Gu, cudaStream_t s);
cudaError_t mr_launch_precond(const Layout1d& lay, int first, int num, const SolveRec* rec,
                              const double* r, double* z, cudaStream_t s);
cudaError_t mr_launch_pcg(const Layout1d& lay, int first, int num, int precision,
                          const double* eta, const double* hx, const double* b, double* x,
                          const SolveRec* given, int kind, double rtol, double rtol_inner,
                          int maxit, int max_refine, SolveRec* rec, void* ws, cudaStream_t s);
cudaError_t mr_launch_rhs(const Layout1d& lay, int first, int num, int precision, double g,
                          const double* eta, const double* u, const double* h,
                          const double* hx, double* f_eta, double* f_U, double* scratch,
                          cudaStream_t s);

struct Layout2d;

// Restarted GMRES(restart) for G x = b, right-preconditioned by A, over every instance of a
// 1d layout (l1, offsets [count + 1]) or the one instance of a 2d layout (l2); vec_len is
// the packed vector length (d P).  coef: per-instance sigma, alpha (and a non-OK status
// that finishes the instance at once); rec: reports (iters = Arnoldi steps, refinements =
// cycles, ratio = final sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b), status).  Host-driven; allocates its
// workspace on the stream and synchronises it before returning.
struct GmresArgs {
  int dim = 1, count = 0;
  const Layout1d* l1 = nullptr;
  const Layout2d* l2 = nullptr;
  const long long* offsets = nullptr;
  long long vec_len = 0;
  const void* tw64 = nullptr;
  const double* eta = nullptr;
  const double* gradh = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  const SolveRec* coef = nullptr;
  SolveRec* rec = nullptr;
  double rtol = 1e-10;
  int restart = 30, maxit = 1000;
};
cudaError_t run_gmres(const GmresArgs& a, cudaStream_t s);

}  // namespace sgn
