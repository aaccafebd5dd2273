// Internal interface of the 2d (doubly periodic) kernels.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "sgn_internal.h"

namespace sgn {

struct Scal2d;   // device-resident scalars of one 2d solve (sgn_2d.cu)

constexpr int kMaxBatch2dAbi = 32;   // instances of one 2d layout (a persistent launch's limit)

// Events around the persistent inner-solve launches of a layout while profiling is on, and
// the inner iterations each launch ran.
struct Prof2d {
  std::vector<cudaEvent_t> a, b;
  std::vector<long long> iters;
};

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
  mutable cudaGraph_t solve_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // sources
  mutable bool solve_graph_off = false;   // building one failed: host-driven solves
  double* stage = nullptr;
  SolveRec* stage_rec = nullptr;
  // Persistent float32 inner solve (sgn_2d_pcg.cu): float32 eta, h_x, h_y (3 planes of P),
  // its instance descriptor (device), per-unit partial sums, the barrier words, the column
  // tile width and the cooperative grid.  inner_form 1 runs the inner iteration as four
  // kernels per iteration instead (k2_cols, k2_rows_matvec, k2_cols, k2_update).
  float* ehh = nullptr;
  void* pinst = nullptr;
  double* pparts = nullptr;
  unsigned* pbar = nullptr;
  int p_tw = 0, p_grid = 0;
  int p_maxb = 3;           // the persistent form's transforms: stages up to radix 2^p_maxb
  int p_gt = 0;             // the persistent form's threads per unit (0: by the unit count)
  int inner_form = 0;
  // non-null while profiling: mixed solves take the host-driven path and bracket each
  // persistent launch with events
  Prof2d* prof = nullptr;
  // Grids whose nx or ny is not a power of two (sgn_2d_mr.cu): full complex spectra,
  // host-driven solves.  Of the buffers above only parts and sc are allocated.
  bool mr = false;
  void* mr_twx = nullptr;      // twiddles of nx: float64, float32, double-float tables
  void* mr_twy = nullptr;      // of ny
  long long mr_lenx = 0, mr_leny = 0;   // entries per table (even)
  void* mr_w = nullptr;        // kMr2dPlanes complex-double planes of P
  double* mr_dev = nullptr;    // dot-product partials and results
  double* mr_host = nullptr;   // pinned copies of the results
  void* mr_sc = nullptr;       // the device-driven solve's scalars
};

// A batch of B >= 2 instances on one grid: B single-instance layouts (instance 0 is the
// layout's own Layout2d, `more` holds instances 1..B-1), per-instance staging of the
// caller's batch-packed fields into the single-instance packing (eta [P], grad h [2P],
// b [2P], x [2P]), and the buffers of the persistent inner solve that advances every
// instance's float32 inner PCG in one launch.
struct Batch2d {
  int B = 0;
  std::vector<Layout2d> more;
  double* stage = nullptr;        // B x 7P
  void* pinst = nullptr;          // d2::PInst2d [B]
  double* pparts = nullptr;       // B (H + ny/2)
  unsigned* pbar = nullptr;
  int p_grid = 0, p_tw = 0;
  Layout2d& inst(Layout2d& first, int b) { return b == 0 ? first : more[b - 1]; }
};

cudaError_t layout2d_create(Layout2d& L, const sgn_grid& g);
// Appends a while node (condition handle h) after the work captured so far on the capturing
// stream cs, which keeps capturing after the node; returns the node's body graph.
cudaError_t capture_add_while(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraph_t* body);
// Destroys a layout's cached solve graphs (executable and source).
void drop_solve_graphs(const Layout2d& L);

// ---- grids with a side that is not a power of two (sgn_2d_mr.cu) --------------------------
// A side n = 2^a 3^b 5^c (a >= 1) with 6 <= n <= 1024.
bool mr2d_side_ok(int n);
cudaError_t mr2d_create(Layout2d& L);
void mr2d_destroy(Layout2d& L);
cudaError_t mr2d_grad(const Layout2d& L, const double* f, double* gradf, cudaStream_t s);
cudaError_t mr2d_apply_G(const Layout2d& L, const double* eta, const double* gradh,
                         const double* u, double* Gu, cudaStream_t s);
cudaError_t mr2d_precond(const Layout2d& L, const SolveRec* rec, const double* r, double* z,
                         cudaStream_t s);
cudaError_t mr2d_pcg(const Layout2d& L, int precision, const double* eta, const double* gradh,
                     const double* b, double* x, const SolveRec* given, int kind, double rtol,
                     double rtol_inner, int maxit, int max_refine, SolveRec* rec,
                     cudaStream_t s);
cudaError_t mr2d_rhs(const Layout2d& L, double g, const double* eta, const double* u,
                     const double* h, const double* gradh, double* f_eta, double* f_U,
                     cudaStream_t s);
cudaError_t batch2d_create(Batch2d& Bt, Layout2d& first, const sgn_grid& g, int B);
void batch2d_destroy(Batch2d& Bt);
// Batched constraint solves of the B instances (fields packed as the ABI's batches: scalar
// instance b at [b P, b P + P), vector components at [b P, ...) and [Ptot + b P, ...)).
// given (nullable): [B] coefficients; rec: [B] reports.  The mixed path runs a host-driven
// refinement loop (two stream synchronisations per pass) around one persistent inner-solve
// launch for every instance that needs a pass; the float64 path solves instance by instance.
cudaError_t launch_pcg2d_batch(Layout2d& first, Batch2d& Bt, const void* tw64, const void* tw32,
                               int precision, const double* eta, const double* gradh,
                               const double* b, double* x, const SolveRec* given, int kind,
                               double rtol, double rtol_inner, int maxit, int max_refine,
                               SolveRec* rec, cudaStream_t s);
// Copies instance b of batch-packed fields into / out of its staging block.
cudaError_t batch2d_stage_in(const Layout2d& L, double* st, int b, long long Ptot,
                             const double* scal, const double* vec0, const double* vec1,
                             const double* vec2, cudaStream_t s);
cudaError_t batch2d_stage_out(const Layout2d& L, const double* stvec, int b, long long Ptot,
                              double* vec, cudaStream_t s);
void layout2d_destroy(Layout2d& L);
size_t layout2d_res_bytes(const Layout2d& L);
// Inner-solve form: 0 the persistent inner solve (default), 1 four kernels per inner
// iteration; tile_width: columns per column tile of the persistent form.  Drops the cached
// solve graphs.
cudaError_t layout2d_set_inner_form(Layout2d& L, int form, int tile_width);
// Largest radix of the persistent form's transform stages, log2 (3: radix 8, 4: radix 16).
// Drops the cached solve graphs when it changes.
cudaError_t layout2d_set_radix(Layout2d& L, int maxb);
cudaError_t layout2d_set_unit_threads(Layout2d& L, int threads);
int persist2d_tile_width(int nx, int ny, int B, int grid);
bool persist2d_tile_ok(int nx, int ny, int tile_width);

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
