// 2d grids whose nx or ny is not a power of two (n = 2^a 3^b 5^c, a >= 1, 6 <= n <= 1024;
// the grids of §6.1 at sizes such as 384 x 240).  Fields keep the [ny][nx] row-major
// packing; spectra are full complex planes [ny][nx] (16 bytes per entry).  A 2d transform
// is a row pass (a CTA transforms a band of rows in shared memory with the mixed-radix
// Stockham FFT of sgn_mr_fft.cuh) and a column pass (a CTA gathers kColTile columns into
// shared memory, transforms them as one batch and scatters them back).  Two real fields
// share one complex transform (f + i g): every operator here is real in physical space, so
// it acts on both parts at once, and a single field's spectrum is recovered from a packed
// one as (Z(k) + conj Z(-k)) / 2 and (Z(k) - conj Z(-k)) / (2i).
//
// Operations, with the same definitions as the power-of-two kernels:
//   grad f                (§6.1: D = F^{-1}(iK)F per axis, Nyquist wavenumbers 0)
//   G u                   (Def:G: eta u - grad(eta^3/3 div u + eta^2/2 grad h.u)
//                          + grad h (eta^2/2 div u + eta grad h.u))
//   A^{-1} r              (Def:A: per mode (sigma I + alpha k k^T)^{-1}, Sherman-Morrison)
//   PCG                   (§3.2 with the stopping rule sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b);
//                          float64, or float32 inner solves inside float64 refinement)
//   right-hand side       (Eq:DAE_DSWE with Def:bigF in 2d, float64)
// A solve runs as one cached graph whose loops are while nodes driven by device-side
// decisions (build_mr_graph); under stream capture the same steps run host-driven.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/sgn.h"
#include "sgn_2d.h"
#include "sgn_2d_dev.cuh"
#include "sgn_mr_fft.cuh"

namespace sgn {
namespace {

using mr::MrPlan;
using mr::mr_plan;

constexpr int kRowNT = 128;            // threads of a row-pass CTA
constexpr int kRowElems = 2048;        // complex entries per row-pass CTA (whole rows)
constexpr int kColNT = 256;            // threads of a column-pass CTA
constexpr int kColTile = 4;            // columns per column-pass CTA
constexpr int kRedBlocks = 256;        // first-stage blocks of a dot product
constexpr int kMaxSide = 1024;
constexpr double kPi2 = 6.283185307179586476925286766559;

// ---- device views -------------------------------------------------------------------------
struct Grid2 {
  int nx, ny;
  long long P;
  double kx, ky;          // 2 pi / Lx, 2 pi / Ly
};

__device__ __forceinline__ double wnum(int j, int n, double unit) {
  const int h = n >> 1;
  return unit * (double)(j < h ? j : (j == h ? 0 : j - n));
}

// the mirror -k of the mode at linear index i = jy nx + jx
__device__ __forceinline__ long long mirror(const Grid2& G, long long i) {
  const int jy = (int)(i / G.nx), jx = (int)(i - (long long)jy * G.nx);
  const int my = jy == 0 ? 0 : G.ny - jy, mx = jx == 0 ? 0 : G.nx - jx;
  return (long long)my * G.nx + mx;
}

template <typename T>
__device__ __forceinline__ T cvt(double v) { return (T)v; }

// ---- transform passes ---------------------------------------------------------------------
// K planes of P entries at stride P: rows of every plane, nb rows per CTA (blockIdx.y: plane)
template <typename T>
__global__ void __launch_bounds__(kRowNT) k2m_rows(cplx<T>* __restrict__ Z, int nx, int ny,
                                                  long long P, int nb, bool inv,
                                                  const cplx<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* a = reinterpret_cast<cplx<T>*>(smem);
  cplx<T>* b = a + (size_t)nb * nx;
  const int y0 = blockIdx.x * nb;
  const int rows = min(nb, ny - y0);
  cplx<T>* base = Z + (long long)blockIdx.y * P + (long long)y0 * nx;
  const int cnt = rows * nx;
  for (int i = threadIdx.x; i < cnt; i += kRowNT) a[i] = base[i];
  __syncthreads();
  MrPlan pl;
  mr_plan(nx, pl);
  const cplx<T>* r = mr::mr_fft<T, kRowNT>(a, b, pl, inv, tw, rows);
  for (int i = threadIdx.x; i < cnt; i += kRowNT) base[i] = r[i];
}

// columns x0 .. x0 + kColTile - 1 of every plane, gathered as kColTile sequences of ny
template <typename T>
__global__ void __launch_bounds__(kColNT) k2m_cols(cplx<T>* __restrict__ Z, int nx, int ny,
                                                  long long P, bool inv,
                                                  const cplx<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* a = reinterpret_cast<cplx<T>*>(smem);
  cplx<T>* b = a + (size_t)kColTile * ny;
  const int x0 = blockIdx.x * kColTile;
  const int cols = min(kColTile, nx - x0);
  cplx<T>* base = Z + (long long)blockIdx.y * P + x0;
  const int cnt = ny * cols;
  for (int i = threadIdx.x; i < cnt; i += kColNT) {
    const int y = i / cols, c = i - y * cols;
    a[c * ny + y] = base[(long long)y * nx + c];
  }
  __syncthreads();
  MrPlan pl;
  mr_plan(ny, pl);
  const cplx<T>* r = mr::mr_fft<T, kColNT>(a, b, pl, inv, tw, cols);
  for (int i = threadIdx.x; i < cnt; i += kColNT) {
    const int y = i / cols, c = i - y * cols;
    base[(long long)y * nx + c] = r[c * ny + y];
  }
}

// ---- spectral kernels (one thread per mode of a full plane) --------------------------------
enum SpecOp { SP_GRAD = 0, SP_DIV = 1, SP_AINV = 2 };

// in: a packed spectrum Z (of f, or of f + i g).  SP_GRAD: out = i kx F - ky F, the packed
// spectrum of (f_x, f_y) of the real field f (Z = F).  SP_DIV: out = i kx U + i ky V, the
// spectrum of u_x + v_y of Z = U + i V.  SP_AINV: out = Z0 + i Z1 with (sigma I + alpha k
// k^T) (Z0, Z1) = (U, V); sigma, alpha from rec.  Scale s multiplies the output (1/P folds
// the inverse transform's normalisation in).
template <typename T, int OP>
__global__ void k2m_spec(Grid2 G, const cplx<T>* __restrict__ Z, cplx<T>* __restrict__ out,
                         const SolveRec* __restrict__ rec, double s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G.P;
       i += (long long)gridDim.x * blockDim.x) {
    const int jy = (int)(i / G.nx), jx = (int)(i - (long long)jy * G.nx);
    const T kx = cvt<T>(wnum(jx, G.nx, G.kx)), ky = cvt<T>(wnum(jy, G.ny, G.ky));
    const T sc = cvt<T>(s);
    const cplx<T> z = Z[i];
    if constexpr (OP == SP_GRAD) {
      // i kx F - ky F
      out[i] = mk((-kx * z.y - ky * z.x) * sc, (kx * z.x - ky * z.y) * sc);
    } else {
      const cplx<T> zm = conj(Z[mirror(G, i)]);
      const T h = cvt<T>(0.5);
      const cplx<T> U = mk((z.x + zm.x) * h, (z.y + zm.y) * h);      // (Z + conj Z(-k)) / 2
      const cplx<T> V = mk((z.y - zm.y) * h, (zm.x - z.x) * h);      // (Z - conj Z(-k)) / 2i
      if constexpr (OP == SP_DIV) {
        // i (kx U + ky V)
        const cplx<T> d = mk(kx * U.x + ky * V.x, kx * U.y + ky * V.y);
        out[i] = mk(-d.y * sc, d.x * sc);
      } else {
        const T sig = cvt<T>(rec->sigma), al = cvt<T>(rec->alpha);
        // z = (r - alpha k (k.r) / (sigma + alpha |k|^2)) / sigma
        const T den = sig + al * (kx * kx + ky * ky);
        const cplx<T> kr = mk(kx * U.x + ky * V.x, kx * U.y + ky * V.y);
        const T f = al / den;
        const cplx<T> Z0 = mk((U.x - f * kx * kr.x) / sig, (U.y - f * kx * kr.y) / sig);
        const cplx<T> Z1 = mk((V.x - f * ky * kr.x) / sig, (V.y - f * ky * kr.y) / sig);
        // Z0 + i Z1
        out[i] = mk((Z0.x - Z1.y) * sc, (Z0.y + Z1.x) * sc);
      }
    }
  }
}

// ---- pointwise kernels ------------------------------------------------------------------
// Z = a + i b (b nullable: 0) in T
template <typename T, typename S>
__global__ void k2m_pack(long long P, const S* __restrict__ a, const S* __restrict__ b,
                         cplx<T>* __restrict__ Z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x)
    Z[i] = mk((T)a[i], b ? (T)b[i] : (T)0);
}

// a = Re Z, b = Im Z (b nullable)
template <typename T, typename S>
__global__ void k2m_unpack(long long P, const cplx<T>* __restrict__ Z, S* __restrict__ a,
                           S* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const cplx<T> z = Z[i];
    a[i] = (S)z.x;
    if (b) b[i] = (S)z.y;
  }
}

// G u, first half: from d = div u (Re Zd) form the pointwise terms.  W = w + 0i with
// w = eta^3/3 d + eta^2/2 s (the field whose gradient G subtracts), and the local parts
// l = eta u + grad h (eta^2/2 d + eta s), s = grad h . u, written to out (2 planes).
template <typename T, typename S>
__global__ void k2m_G_mid(long long P, const double* __restrict__ eta,
                          const double* __restrict__ gh, const S* __restrict__ u,
                          const cplx<T>* __restrict__ Zd, cplx<T>* __restrict__ W,
                          T* __restrict__ l) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const T e = (T)eta[i], hx = (T)gh[i], hy = (T)gh[P + i];
    const T u0 = (T)u[i], u1 = (T)u[P + i];
    const T d = Zd[i].x;
    const T sv = hx * u0 + hy * u1;
    const T e2h = e * e * (T)0.5;
    W[i] = mk(e * e * e * (T)(1.0 / 3.0) * d + e2h * sv, (T)0);
    const T c = e2h * d + e * sv;
    l[i] = e * u0 + hx * c;
    l[P + i] = e * u1 + hy * c;
  }
}

// G u, second half: out = l - grad w (grad w packed in Zg)
template <typename T, typename S>
__global__ void k2m_G_end(long long P, const T* __restrict__ l, const cplx<T>* __restrict__ Zg,
                          S* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const cplx<T> g = Zg[i];
    out[i] = (S)(l[i] - g.x);
    out[P + i] = (S)(l[P + i] - g.y);
  }
}

// ---- deterministic dot products ---------------------------------------------------------
// partial sums over a fixed grid (block b takes a fixed set of indices, fixed tree), then one
// block adds the partials in order: the result does not depend on timing.
template <typename S>
__global__ void __launch_bounds__(256) k2m_dot1(long long n, const S* __restrict__ a,
                                               const S* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[256 / 32 + 1];
  double v = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * kRedBlocks)
    v += (double)a[i] * (double)b[i];
  v = block_sum<256>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(256) k2m_dot2(const double* __restrict__ part,
                                               double* __restrict__ out) {
  __shared__ double red[256 / 32 + 1];
  double v = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += 256) v += part[i];
  v = block_sum<256>(v, red);
  if (threadIdx.x == 0) *out = v;
}

// y = a x + y (float64 scalar from the host), in S
template <typename S>
__global__ void k2m_axpy(long long n, double a, const S* __restrict__ x, S* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (S)((double)y[i] + a * (double)x[i]);
}

// p = z + beta p
template <typename S>
__global__ void k2m_xpby(long long n, const S* __restrict__ z, double beta, S* __restrict__ p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = (S)((double)z[i] + beta * (double)p[i]);
}

// out = a - b (float64) scaled into S: out = s (a - b)
template <typename S>
__global__ void k2m_sub_scale(long long n, const double* __restrict__ a,
                              const double* __restrict__ b, double s, S* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (S)(s * (a[i] - b[i]));
}

// x += s d (d float32)
__global__ void k2m_correct(long long n, double s, const float* __restrict__ d,
                            double* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += s * (double)d[i];
}

// out = s a, converted to S
template <typename S>
__global__ void k2m_scale_to(long long n, double s, const double* __restrict__ a,
                             S* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (S)(s * a[i]);
}

// the solve report (coefficients kept)
__global__ void k2m_report(SolveRec* rec, int iters, int refinements, double ratio, int status) {
  rec->iters = iters;
  rec->refinements = refinements;
  rec->ratio = ratio;
  rec->status = status;
}

// ---- device-driven solve: scalars and decisions -------------------------------------------
// The cached solve graph keeps every decision on the device: the while nodes' conditions are
// set by the kernels below from these scalars (options written before each launch).
struct MrScal {
  double rtol, rtol_in;       // options
  int maxit, max_refine, kind;
  double bb, rz, rzn, pq, alpha, beta, tol, nr, scale, ratio;
  int iters, refinements, status, st_in, it0, skip, zero_x, nofit;
};

__global__ void k2m_opts(MrScal* S, double rtol, double rtol_in, int maxit, int max_refine) {
  S->rtol = rtol;
  S->rtol_in = rtol_in;
  S->maxit = maxit;
  S->max_refine = max_refine;
}

// after the coefficients (rec) and b.A^{-1}b: start the solve, or finish it at once
__global__ void k2m_begin(MrScal* S, const SolveRec* rec) {
  S->iters = 0;
  S->refinements = 0;
  S->ratio = 0.0;
  S->st_in = SGN_OK;
  S->skip = 0;
  S->zero_x = 0;
  S->nofit = 0;
  S->status = rec->status;
  if (S->status != SGN_OK) {         // reported by the coefficients; x untouched
    S->skip = 1;
    S->nofit = 1;
    return;
  }
  const double bb = S->bb;
  if (!(bb > 0.0)) {                 // x = 0: b = 0 solves exactly, a non-finite b breaks down
    S->zero_x = 1;
    S->skip = 1;
    S->status = bb == 0.0 ? SGN_OK : SGN_ERR_BREAKDOWN;
  }
}

// float64 PCG: after r.z of the first residual; the loop runs while sqrt(rz) > tol
__global__ void k2m_init64(MrScal* S, cudaGraphConditionalHandle h) {
  unsigned go = 0u;
  if (!S->skip) {
    S->tol = S->rtol * sqrt(S->bb);
    if (sqrt(S->rz) > S->tol) {
      if (S->iters >= S->maxit) S->status = SGN_ERR_NOT_CONVERGED;
      else go = 1u;
    }
  }
  cudaGraphSetConditional(h, go);
}

// alpha = rz / p.Gp, or a breakdown (skip marks the rest of the iteration)
__global__ void k2m_alpha(MrScal* S, int inner) {
  if (S->skip) return;
  const double pq = S->pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (inner) S->st_in = SGN_ERR_BREAKDOWN;
    else S->status = SGN_ERR_BREAKDOWN;
    S->skip = 1;
    return;
  }
  S->alpha = S->rz / pq;
}

// beta = rz_new / rz and the loop condition (float64 PCG: tol; inner PCG: tin)
__global__ void k2m_beta(MrScal* S, int inner, cudaGraphConditionalHandle h) {
  unsigned go = 0u;
  if (!S->skip) {
    S->iters += 1;
    const double rzn = S->rzn;
    if (!isfinite(rzn)) {
      if (inner) S->st_in = SGN_ERR_BREAKDOWN;
      else S->status = SGN_ERR_BREAKDOWN;
      S->skip = 1;
    } else {
      S->beta = rzn / S->rz;
      S->rz = rzn;
      if (sqrt(rzn) > S->tol) {
        if (S->iters >= S->maxit) {
          if (inner) S->st_in = SGN_ERR_NOT_CONVERGED;
          else S->status = SGN_ERR_NOT_CONVERGED;
        } else {
          go = 1u;
        }
      }
    }
  }
  cudaGraphSetConditional(h, go);
}

// mixed: after a refinement residual's r.A^{-1}r (in rz): done, out of budget, or the next
// inner solve (its tolerance and the scale of r)
__global__ void k2m_decide(MrScal* S, cudaGraphConditionalHandle h) {
  unsigned go = 0u;
  if (!S->zero_x && !S->nofit) {
    const double nr = sqrt(fmax(S->rz, 0.0));
    S->ratio = nr / sqrt(S->bb);
    if (S->ratio <= S->rtol) {
      S->status = SGN_OK;
    } else if (S->status != SGN_OK) {
      // a float32 breakdown without progress ended the solve
    } else if (!isfinite(nr)) {
      S->status = SGN_ERR_BREAKDOWN;
    } else if (S->refinements >= S->max_refine || S->iters >= S->maxit) {
      S->status = SGN_ERR_NOT_CONVERGED;
    } else {
      S->nr = nr;
      S->scale = 1.0 / nr;
      S->tol = S->rtol_in > 0.0 ? S->rtol_in : fmin(0.1, fmax(1e-6, 0.3 * S->rtol / S->ratio));
      go = 1u;
    }
  }
  cudaGraphSetConditional(h, go);
}

// mixed: the inner solve starts from d = 0 with r.z in rz
__global__ void k2m_inner_init(MrScal* S, cudaGraphConditionalHandle h) {
  S->it0 = S->iters;
  S->st_in = SGN_OK;
  S->skip = 0;
  unsigned go = 0u;
  if (sqrt(fmax(S->rz, 0.0)) > S->tol) {
    if (S->iters >= S->maxit) S->st_in = SGN_ERR_NOT_CONVERGED;
    else go = 1u;
  }
  cudaGraphSetConditional(h, go);
}

// mixed: after an inner solve; a float32 breakdown without progress ends the solve
__global__ void k2m_after_inner(MrScal* S) {
  if (S->st_in == SGN_ERR_BREAKDOWN && S->iters == S->it0) S->status = SGN_ERR_BREAKDOWN;
  S->refinements += 1;
  S->skip = 0;
}

// y += sign alpha x, p = z + beta p, x += nr d, out = scale r: the loop's vector updates with
// their scalars read on the device (skipped after a breakdown in the same iteration)
template <typename Sv>
__global__ void k2m_axpy_s(long long n, const MrScal* S, double sign, const Sv* __restrict__ x,
                           Sv* __restrict__ y) {
  if (S->skip) return;
  const double a = sign * S->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (Sv)((double)y[i] + a * (double)x[i]);
}

template <typename Sv>
__global__ void k2m_xpby_s(long long n, const MrScal* S, const Sv* __restrict__ z,
                           Sv* __restrict__ p) {
  if (S->skip) return;
  const double b = S->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = (Sv)((double)z[i] + b * (double)p[i]);
}

__global__ void k2m_correct_s(long long n, const MrScal* S, const float* __restrict__ d,
                              double* __restrict__ x) {
  const double s = S->nr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += s * (double)d[i];
}

__global__ void k2m_scale_s(long long n, const MrScal* S, const double* __restrict__ r,
                            float* __restrict__ out) {
  const double s = S->scale;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)(s * r[i]);
}

// the report into rec (coefficients kept); x = 0 when b was zero (or not finite)
__global__ void k2m_finish(const MrScal* S, SolveRec* rec, double* __restrict__ x, long long n,
                           int mixed) {
  if (S->zero_x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      x[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rec->iters = S->iters;
    rec->refinements = S->refinements;
    rec->status = S->status;
    rec->ratio = (S->zero_x || S->nofit)
                     ? 0.0
                     : (mixed ? S->ratio : sqrt(fmax(S->rz, 0.0)) / sqrt(S->bb));
  }
}

// the coefficient kind of the captured coefficient step (k2_coeffs reads it from sc)
__global__ void k2m_kind(Scal2d* sc, int kind) { sc->kind = kind; }

// given coefficients: rec = given with status OK
__global__ void k2m_given(const SolveRec* given, SolveRec* rec) {
  SolveRec r = *given;
  r.status = SGN_OK;
  *rec = r;
}

// ---- right-hand side (Eq:DAE_DSWE with Def:bigF, 2d; reading R6) -------------------------
// products whose divergence or gradient the right-hand side takes
__global__ void k2m_rhs_pre(long long P, const double* __restrict__ eta,
                            const double* __restrict__ u, const double* __restrict__ h,
                            const double* __restrict__ gh, double* __restrict__ s,
                            double* __restrict__ eu, double* __restrict__ ev,
                            double* __restrict__ zeta, double* __restrict__ fu,
                            double* __restrict__ fuv, double* __restrict__ fv) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const double e = eta[i], uu = u[i], vv = u[P + i];
    s[i] = gh[i] * uu + gh[P + i] * vv;
    eu[i] = e * uu;
    ev[i] = e * vv;
    zeta[i] = e - h[i];
    fu[i] = e * uu * uu;
    fuv[i] = e * uu * vv;
    fv[i] = e * vv * vv;
  }
}

// Phi = eta^3 Q/3 + eta^2 m d + eta^2 S/2 + eta m s, Psi = eta^2 Q/2 + eta m d + eta S + m s
// with S = u.grad s, Q = u.grad d - d^2
__global__ void k2m_rhs_mid(long long P, const double* __restrict__ eta,
                            const double* __restrict__ u, const double* __restrict__ d,
                            const double* __restrict__ m, const double* __restrict__ s,
                            const double* __restrict__ sx, const double* __restrict__ sy,
                            const double* __restrict__ dx, const double* __restrict__ dy,
                            double* __restrict__ Phi, double* __restrict__ Psi) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const double e = eta[i], uu = u[i], vv = u[P + i];
    const double dd = d[i], mm = m[i], ss = s[i];
    const double S = uu * sx[i] + vv * sy[i];
    const double Q = uu * dx[i] + vv * dy[i] - dd * dd;
    const double e2 = e * e;
    Phi[i] = e2 * e * Q / 3.0 + e2 * mm * dd + e2 * S / 2.0 + e * mm * ss;
    Psi[i] = e2 * Q / 2.0 + e * mm * dd + e * S + mm * ss;
  }
}

// f_eta = -m; f_U = -g eta grad zeta - div(eta u u^T) + grad Phi - grad h Psi
__global__ void k2m_rhs_end(long long P, double g, const double* __restrict__ eta,
                            const double* __restrict__ gh, const double* __restrict__ m,
                            const double* __restrict__ zx, const double* __restrict__ zy,
                            const double* __restrict__ a1, const double* __restrict__ a2,
                            const double* __restrict__ px, const double* __restrict__ py,
                            const double* __restrict__ Psi, double* __restrict__ f_eta,
                            double* __restrict__ f_U) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const double e = eta[i];
    f_eta[i] = -m[i];
    f_U[i] = -g * e * zx[i] - a1[i] + px[i] - gh[i] * Psi[i];
    f_U[P + i] = -g * e * zy[i] - a2[i] + py[i] - gh[P + i] * Psi[i];
  }
}

// e^{-2 pi i r k / (p R)} tables as in the 1d generic kernels
using mr::k_mr_twiddles;

constexpr int kMr2dPlanes = 14;        // 2 transform planes + 12 work planes (24 real)
constexpr int kScal = 8;               // result slots of the dot products

int blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// ---- host view of a layout's generic buffers ----------------------------------------------
struct Mr {
  const Layout2d& L;
  Grid2 G;
  cplx<double>* A;        // transform planes
  cplx<double>* B;
  double* real0;          // 24 real planes of P doubles
  explicit Mr(const Layout2d& l) : L(l) {
    G.nx = L.nx;
    G.ny = L.ny;
    G.P = L.P;
    G.kx = kPi2 / L.Lx;
    G.ky = kPi2 / L.Ly;
    A = static_cast<cplx<double>*>(L.mr_w);
    B = A + L.P;
    real0 = reinterpret_cast<double*>(A + 2 * L.P);
  }
  double* rp(int j) const { return real0 + (long long)j * L.P; }
  float* fp(int j) const { return reinterpret_cast<float*>(rp(j)); }   // 2P floats
  template <typename T>
  cplx<T>* za() const { return reinterpret_cast<cplx<T>*>(A); }
  template <typename T>
  cplx<T>* zb() const { return reinterpret_cast<cplx<T>*>(B); }
  template <typename T>
  const cplx<T>* twx() const;
  template <typename T>
  const cplx<T>* twy() const;
};
template <>
const cplx<double>* Mr::twx<double>() const { return static_cast<const cplx<double>*>(L.mr_twx); }
template <>
const cplx<double>* Mr::twy<double>() const { return static_cast<const cplx<double>*>(L.mr_twy); }
template <>
const cplx<float>* Mr::twx<float>() const {
  return reinterpret_cast<const cplx<float>*>(static_cast<const char*>(L.mr_twx) + 16 * L.mr_lenx);
}
template <>
const cplx<float>* Mr::twy<float>() const {
  return reinterpret_cast<const cplx<float>*>(static_cast<const char*>(L.mr_twy) + 16 * L.mr_leny);
}

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
  return raise_smem(kernel, bytes);
}

// 2d transform of K planes at Z (stride P); the inverse without the 1/P
template <typename T>
cudaError_t fft2(const Mr& M, cplx<T>* Z, int K, bool inv, cudaStream_t s) {
  const int nx = M.G.nx, ny = M.G.ny;
  const int nb = max(1, kRowElems / nx);
  size_t sm = (size_t)2 * nb * nx * sizeof(cplx<T>);
  cudaError_t e = smem_attr(k2m_rows<T>, sm);
  if (e) return e;
  k2m_rows<T><<<dim3((ny + nb - 1) / nb, K), kRowNT, sm, s>>>(Z, nx, ny, M.G.P, nb, inv,
                                                             M.twx<T>());
  if ((e = cudaGetLastError())) return e;
  sm = (size_t)2 * kColTile * ny * sizeof(cplx<T>);
  if ((e = smem_attr(k2m_cols<T>, sm))) return e;
  k2m_cols<T><<<dim3((nx + kColTile - 1) / kColTile, K), kColNT, sm, s>>>(Z, nx, ny, M.G.P, inv,
                                                                         M.twy<T>());
  return cudaGetLastError();
}

// (f_x, f_y) of the real field f (float64)
cudaError_t grad2(const Mr& M, const double* f, double* fx, double* fy, cudaStream_t s) {
  const long long P = M.G.P;
  const int nb = blocks_for(P);
  k2m_pack<double, double><<<nb, 256, 0, s>>>(P, f, nullptr, M.A);
  cudaError_t e = cudaGetLastError();
  if (!e) e = fft2<double>(M, M.A, 1, false, s);
  if (e) return e;
  k2m_spec<double, SP_GRAD><<<nb, 256, 0, s>>>(M.G, M.A, M.B, nullptr, 1.0 / (double)P);
  if ((e = cudaGetLastError()) || (e = fft2<double>(M, M.B, 1, true, s))) return e;
  k2m_unpack<double, double><<<nb, 256, 0, s>>>(P, M.B, fx, fy);
  return cudaGetLastError();
}

// a_x + b_y of the real fields a, b (float64)
cudaError_t div2(const Mr& M, const double* a, const double* b, double* out, cudaStream_t s) {
  const long long P = M.G.P;
  const int nb = blocks_for(P);
  k2m_pack<double, double><<<nb, 256, 0, s>>>(P, a, b, M.A);
  cudaError_t e = cudaGetLastError();
  if (!e) e = fft2<double>(M, M.A, 1, false, s);
  if (e) return e;
  k2m_spec<double, SP_DIV><<<nb, 256, 0, s>>>(M.G, M.A, M.B, nullptr, 1.0 / (double)P);
  if ((e = cudaGetLastError()) || (e = fft2<double>(M, M.B, 1, true, s))) return e;
  k2m_unpack<double, double><<<nb, 256, 0, s>>>(P, M.B, out, (double*)nullptr);
  return cudaGetLastError();
}

// out = G u in T (u, out: 2 planes of S); l: 2P T of scratch
template <typename T, typename S>
cudaError_t applyG(const Mr& M, const double* eta, const double* gh, const S* u, S* out, T* l,
                   cudaStream_t s) {
  const long long P = M.G.P;
  const int nb = blocks_for(P);
  cplx<T>* A = M.za<T>();
  cplx<T>* B = M.zb<T>();
  k2m_pack<T, S><<<nb, 256, 0, s>>>(P, u, u + P, A);
  cudaError_t e = cudaGetLastError();
  if (!e) e = fft2<T>(M, A, 1, false, s);
  if (e) return e;
  k2m_spec<T, SP_DIV><<<nb, 256, 0, s>>>(M.G, A, B, nullptr, 1.0 / (double)P);
  if ((e = cudaGetLastError()) || (e = fft2<T>(M, B, 1, true, s))) return e;
  k2m_G_mid<T, S><<<nb, 256, 0, s>>>(P, eta, gh, u, B, A, l);
  if ((e = cudaGetLastError()) || (e = fft2<T>(M, A, 1, false, s))) return e;
  k2m_spec<T, SP_GRAD><<<nb, 256, 0, s>>>(M.G, A, B, nullptr, 1.0 / (double)P);
  if ((e = cudaGetLastError()) || (e = fft2<T>(M, B, 1, true, s))) return e;
  k2m_G_end<T, S><<<nb, 256, 0, s>>>(P, l, B, out);
  return cudaGetLastError();
}

// z = A^{-1} r in T (2 planes of S each)
template <typename T, typename S>
cudaError_t ainv(const Mr& M, const SolveRec* rec, const S* r, S* z, cudaStream_t s) {
  const long long P = M.G.P;
  const int nb = blocks_for(P);
  cplx<T>* A = M.za<T>();
  cplx<T>* B = M.zb<T>();
  k2m_pack<T, S><<<nb, 256, 0, s>>>(P, r, r + P, A);
  cudaError_t e = cudaGetLastError();
  if (!e) e = fft2<T>(M, A, 1, false, s);
  if (e) return e;
  k2m_spec<T, SP_AINV><<<nb, 256, 0, s>>>(M.G, A, B, rec, 1.0 / (double)P);
  if ((e = cudaGetLastError()) || (e = fft2<T>(M, B, 1, true, s))) return e;
  k2m_unpack<T, S><<<nb, 256, 0, s>>>(P, B, z, z + P);
  return cudaGetLastError();
}

// the dot product a.b (n entries of S) into result slot k (device)
template <typename S>
cudaError_t dot_to(const Mr& M, const S* a, const S* b, long long n, int k, cudaStream_t s) {
  k2m_dot1<S><<<kRedBlocks, 256, 0, s>>>(n, a, b, M.L.mr_dev);
  k2m_dot2<<<1, 256, 0, s>>>(M.L.mr_dev, M.L.mr_dev + kRedBlocks + k);
  return cudaGetLastError();
}

// result slots [0, k) to the host (synchronises the stream)
cudaError_t read_slots(const Mr& M, int k, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(M.L.mr_host, M.L.mr_dev + kRedBlocks, sizeof(double) * k,
                                  cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

bool mr2d_side_ok(int n) {
  MrPlan P;
  return n >= 6 && n <= kMaxSide && mr_plan(n, P);
}

cudaError_t mr2d_create(Layout2d& L) {
  L.mr = true;
  cudaError_t e;
  auto tables = [&](int n, void** tw, long long* len) -> cudaError_t {
    *len = (n - 1) + ((n - 1) & 1);          // even: the double-float table 16-byte aligned
    cudaError_t r = cudaMalloc(tw, (size_t)40 * *len);
    if (r) return r;
    char* b = static_cast<char*>(*tw);
    k_mr_twiddles<<<(n + 255) / 256, 256>>>(n, reinterpret_cast<cplx<double>*>(b),
                                            reinterpret_cast<cplx<float>*>(b + 16 * *len),
                                            reinterpret_cast<cplx<df>*>(b + 24 * *len));
    return cudaGetLastError();
  };
  if ((e = tables(L.nx, &L.mr_twx, &L.mr_lenx))) return e;
  if ((e = tables(L.ny, &L.mr_twy, &L.mr_leny))) return e;
  if ((e = cudaMalloc(&L.mr_w, (size_t)16 * L.P * kMr2dPlanes))) return e;
  if ((e = cudaMalloc(&L.mr_dev, sizeof(double) * (kRedBlocks + kScal)))) return e;
  if ((e = cudaMallocHost(&L.mr_host, sizeof(double) * kScal))) return e;
  if ((e = cudaMalloc(&L.mr_sc, sizeof(MrScal)))) return e;
  if ((e = cudaMalloc(&L.stage, sizeof(double) * 7 * L.P))) return e;
  if ((e = cudaMalloc(&L.stage_rec, sizeof(SolveRec) * 2))) return e;
  return cudaStreamSynchronize(nullptr);          // the tables (legacy stream)
}

void mr2d_destroy(Layout2d& L) {
  cudaFree(L.mr_twx);
  cudaFree(L.mr_twy);
  cudaFree(L.mr_w);
  cudaFree(L.mr_dev);
  cudaFree(L.mr_sc);
  L.mr_sc = nullptr;
  if (L.mr_host) cudaFreeHost(L.mr_host);
  L.mr_twx = L.mr_twy = L.mr_w = nullptr;
  L.mr_dev = L.mr_host = nullptr;
}

cudaError_t mr2d_grad(const Layout2d& L, const double* f, double* gradf, cudaStream_t s) {
  const Mr M(L);
  return grad2(M, f, gradf, gradf + L.P, s);
}

cudaError_t mr2d_apply_G(const Layout2d& L, const double* eta, const double* gradh,
                         const double* u, double* Gu, cudaStream_t s) {
  const Mr M(L);
  return applyG<double, double>(M, eta, gradh, u, Gu, M.rp(8), s);
}

cudaError_t mr2d_precond(const Layout2d& L, const SolveRec* rec, const double* r, double* z,
                         cudaStream_t s) {
  const Mr M(L);
  return ainv<double, double>(M, rec, r, z, s);
}

namespace {

// The solve as one graph (inputs from L.stage, options from the scalars, the report to
// L.stage_rec[1]): the float64 PCG loop, or the refinement loop around the float32 inner
// loop, as while nodes whose conditions the decision kernels set.
cudaError_t build_mr_graph(const Layout2d& L, bool mixed, bool given, cudaGraphExec_t* out,
                           cudaGraph_t* src) {
  const Mr M(L);
  const long long P = L.P, V = 2 * P;
  const int nb = blocks_for(V);
  MrScal* S = static_cast<MrScal*>(L.mr_sc);
  const double* eta = L.stage;
  const double* gh = L.stage + P;
  const double* b = L.stage + 3 * P;
  double* x = L.stage + 5 * P;
  SolveRec* rec = L.stage_rec + 1;
  double* r = M.rp(0);
  double* p = M.rp(2);
  double* z = M.rp(4);
  double* q = M.rp(6);
  double* l = M.rp(8);
  float* rf = M.fp(10);
  float* pf = M.fp(11);
  float* zf = M.fp(12);
  float* qf = M.fp(13);
  float* df_ = M.fp(14);
  float* lf = M.fp(15);
  cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaSuccess;
  int capturing = 0;
  for (auto& c : cs)
    if (!e) e = cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking);
  if (!e) e = cudaGraphCreate(&g, 0);
  auto begin = [&](int i, cudaGraph_t into) {
    cudaError_t r_ = cudaStreamBeginCaptureToGraph(cs[i], into, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed);
    if (!r_) capturing |= 1 << i;
    return r_;
  };
  auto end = [&](int i) {
    cudaGraph_t dummy;
    capturing &= ~(1 << i);
    cudaError_t r_ = cudaStreamEndCapture(cs[i], &dummy);
    return r_ ? r_ : cudaGetLastError();
  };
  auto last = [&]() { return cudaGetLastError(); };
  // r = b - G x, z = A^{-1} r, rz = r.z (float64) on stream st
  auto residual64 = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t r_ = applyG<double, double>(M, eta, gh, x, q, l, st);
    if (r_) return r_;
    k2m_sub_scale<double><<<nb, 256, 0, st>>>(V, b, q, 1.0, r);
    if ((r_ = last()) || (r_ = ainv<double, double>(M, rec, r, z, st))) return r_;
    k2m_dot1<double><<<kRedBlocks, 256, 0, st>>>(V, r, z, L.mr_dev);
    k2m_dot2<<<1, 256, 0, st>>>(L.mr_dev, &S->rz);
    return last();
  };
  if (!e) e = begin(0, g);
  if (!e) {
    if (given) k2m_given<<<1, 1, 0, cs[0]>>>(L.stage_rec, rec);
    e = last();
    if (!e && !given) e = launch_coeffs2d(L, eta, gh, -1, rec, cs[0]);
  }
  // b.A^{-1}b, then the start decisions
  if (!e) e = ainv<double, double>(M, rec, b, z, cs[0]);
  if (!e) {
    k2m_dot1<double><<<kRedBlocks, 256, 0, cs[0]>>>(V, b, z, L.mr_dev);
    k2m_dot2<<<1, 256, 0, cs[0]>>>(L.mr_dev, &S->bb);
    k2m_begin<<<1, 1, 0, cs[0]>>>(S, rec);
    e = last();
  }
  if (!mixed) {
    cudaGraphConditionalHandle hin;
    cudaGraph_t body = nullptr;
    if (!e) e = residual64(cs[0]);
    if (!e) e = cudaMemcpyAsync(p, z, sizeof(double) * V, cudaMemcpyDeviceToDevice, cs[0]);
    if (!e) e = cudaGraphConditionalHandleCreate(&hin, g, 0, 0);
    if (!e) {
      k2m_init64<<<1, 1, 0, cs[0]>>>(S, hin);
      e = last();
    }
    if (!e) e = capture_add_while(cs[0], hin, &body);
    if (!e) e = begin(1, body);
    if (!e) e = applyG<double, double>(M, eta, gh, p, q, l, cs[1]);
    if (!e) {
      k2m_dot1<double><<<kRedBlocks, 256, 0, cs[1]>>>(V, p, q, L.mr_dev);
      k2m_dot2<<<1, 256, 0, cs[1]>>>(L.mr_dev, &S->pq);
      k2m_alpha<<<1, 1, 0, cs[1]>>>(S, 0);
      k2m_axpy_s<double><<<nb, 256, 0, cs[1]>>>(V, S, 1.0, p, x);
      k2m_axpy_s<double><<<nb, 256, 0, cs[1]>>>(V, S, -1.0, q, r);
      e = last();
    }
    if (!e) e = ainv<double, double>(M, rec, r, z, cs[1]);
    if (!e) {
      k2m_dot1<double><<<kRedBlocks, 256, 0, cs[1]>>>(V, r, z, L.mr_dev);
      k2m_dot2<<<1, 256, 0, cs[1]>>>(L.mr_dev, &S->rzn);
      k2m_beta<<<1, 1, 0, cs[1]>>>(S, 0, hin);
      k2m_xpby_s<double><<<nb, 256, 0, cs[1]>>>(V, S, z, p);
      e = last();
    }
    if (!e) e = end(1);
  } else {
    cudaGraphConditionalHandle hout, hin;
    cudaGraph_t body = nullptr, ibody = nullptr;
    if (!e) e = residual64(cs[0]);
    if (!e) e = cudaGraphConditionalHandleCreate(&hout, g, 0, 0);
    if (!e) {
      k2m_decide<<<1, 1, 0, cs[0]>>>(S, hout);
      e = last();
    }
    if (!e) e = capture_add_while(cs[0], hout, &body);
    if (!e) e = begin(1, body);
    // the inner solve of G d = r / ||r|| from d = 0
    if (!e) {
      k2m_scale_s<<<nb, 256, 0, cs[1]>>>(V, S, r, rf);
      e = last();
    }
    if (!e) e = cudaMemsetAsync(df_, 0, sizeof(float) * V, cs[1]);
    if (!e) e = ainv<float, float>(M, rec, rf, zf, cs[1]);
    if (!e) e = cudaMemcpyAsync(pf, zf, sizeof(float) * V, cudaMemcpyDeviceToDevice, cs[1]);
    if (!e) e = cudaGraphConditionalHandleCreate(&hin, body, 0, 0);
    if (!e) {
      k2m_dot1<float><<<kRedBlocks, 256, 0, cs[1]>>>(V, rf, zf, L.mr_dev);
      k2m_dot2<<<1, 256, 0, cs[1]>>>(L.mr_dev, &S->rz);
      k2m_inner_init<<<1, 1, 0, cs[1]>>>(S, hin);
      e = last();
    }
    if (!e) e = capture_add_while(cs[1], hin, &ibody);
    if (!e) e = begin(2, ibody);
    if (!e) e = applyG<float, float>(M, eta, gh, pf, qf, lf, cs[2]);
    if (!e) {
      k2m_dot1<float><<<kRedBlocks, 256, 0, cs[2]>>>(V, pf, qf, L.mr_dev);
      k2m_dot2<<<1, 256, 0, cs[2]>>>(L.mr_dev, &S->pq);
      k2m_alpha<<<1, 1, 0, cs[2]>>>(S, 1);
      k2m_axpy_s<float><<<nb, 256, 0, cs[2]>>>(V, S, 1.0, pf, df_);
      k2m_axpy_s<float><<<nb, 256, 0, cs[2]>>>(V, S, -1.0, qf, rf);
      e = last();
    }
    if (!e) e = ainv<float, float>(M, rec, rf, zf, cs[2]);
    if (!e) {
      k2m_dot1<float><<<kRedBlocks, 256, 0, cs[2]>>>(V, rf, zf, L.mr_dev);
      k2m_dot2<<<1, 256, 0, cs[2]>>>(L.mr_dev, &S->rzn);
      k2m_beta<<<1, 1, 0, cs[2]>>>(S, 1, hin);
      k2m_xpby_s<float><<<nb, 256, 0, cs[2]>>>(V, S, zf, pf);
      e = last();
    }
    if (!e) e = end(2);
    if (!e) {
      k2m_after_inner<<<1, 1, 0, cs[1]>>>(S);
      k2m_correct_s<<<nb, 256, 0, cs[1]>>>(V, S, df_, x);
      e = last();
    }
    if (!e) e = residual64(cs[1]);
    if (!e) {
      k2m_decide<<<1, 1, 0, cs[1]>>>(S, hout);
      e = last();
    }
    if (!e) e = end(1);
  }
  if (!e) {
    k2m_finish<<<nb, 256, 0, cs[0]>>>(S, rec, x, V, mixed ? 1 : 0);
    e = last();
  }
  if (!e) e = end(0);
  for (int i = 2; i >= 0; --i)
    if (capturing & (1 << i)) end(i);          // a failed build: close its captures
  if (!e) e = cudaGraphInstantiate(out, g, 0);
  for (auto& c : cs)
    if (c) cudaStreamDestroy(c);
  // as for the power-of-two solve graphs: a graph whose build failed is left alone
  if (!e) *src = g;
  return e;
}

}  // namespace

cudaError_t mr2d_pcg(const Layout2d& L, int precision, const double* eta, const double* gradh,
                     const double* b, double* x, const SolveRec* given, int kind, double rtol,
                     double rtol_inner, int maxit, int max_refine, SolveRec* rec,
                     cudaStream_t s) {
  const Mr M(L);
  const long long P = L.P, V = 2 * P;
  const int nb = blocks_for(V);
  cudaError_t e;
  // ---- device-driven: one graph launch between staging copies
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (!L.solve_graph_off && cudaStreamIsCapturing(s, &cst) == cudaSuccess &&
      cst == cudaStreamCaptureStatusNone) {
    const int mi = precision == SGN_PREC_MIXED ? 1 : 0, gi = given ? 1 : 0;
    cudaGraphExec_t& ex = L.solve_exec[mi][gi];
    if (!ex && build_mr_graph(L, mi == 1, gi == 1, &ex, &L.solve_graph[mi][gi]) != cudaSuccess) {
      cudaGetLastError();
      ex = nullptr;
      L.solve_graph_off = true;
    }
    if (ex) {
      const size_t d = sizeof(double);
      if ((e = cudaMemcpyAsync(L.stage, eta, d * P, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + P, gradh, d * V, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + 3 * P, b, d * V, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + 5 * P, x, d * V, cudaMemcpyDeviceToDevice, s)))
        return e;
      if (given && (e = cudaMemcpyAsync(L.stage_rec, given, sizeof(SolveRec),
                                        cudaMemcpyDeviceToDevice, s)))
        return e;
      k2m_opts<<<1, 1, 0, s>>>(static_cast<MrScal*>(L.mr_sc), rtol, rtol_inner, maxit,
                               max_refine > 0 ? max_refine : 12);
      k2m_kind<<<1, 1, 0, s>>>(L.sc, kind);
      if ((e = cudaGetLastError()) || (e = cudaGraphLaunch(ex, s))) return e;
      if ((e = cudaMemcpyAsync(x, L.stage + 5 * P, d * V, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(rec, L.stage_rec + 1, sizeof(SolveRec), cudaMemcpyDeviceToDevice,
                               s)))
        return e;
      return cudaSuccess;
    }
  }
  // ---- host-driven
  // a1: the coefficients (or the caller's) into rec
  if (given) {
    if ((e = cudaMemcpyAsync(rec, given, sizeof(SolveRec), cudaMemcpyDeviceToDevice, s)))
      return e;
    k2m_report<<<1, 1, 0, s>>>(rec, 0, 0, 0.0, SGN_OK);
    if ((e = cudaGetLastError())) return e;
  } else if ((e = launch_coeffs2d(L, eta, gradh, kind, rec, s))) {
    return e;
  }
  SolveRec R;
  static_assert(sizeof(SolveRec) <= sizeof(double) * kScal, "record fits the pinned slots");
  if ((e = cudaMemcpyAsync(L.mr_host, rec, sizeof(SolveRec), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return e;
  memcpy(&R, L.mr_host, sizeof(SolveRec));
  if (R.status != SGN_OK) return cudaSuccess;       // reported by the coefficients
  double* r = M.rp(0);
  double* p = M.rp(2);
  double* z = M.rp(4);
  double* q = M.rp(6);
  double* l = M.rp(8);
  const double* H = L.mr_host;
  // b.A^{-1}b
  if ((e = ainv<double, double>(M, rec, b, z, s)) || (e = dot_to(M, b, z, V, 0, s)) ||
      (e = read_slots(M, 1, s)))
    return e;
  const double bb = H[0];
  int iters = 0, refinements = 0, status = SGN_OK;
  double ratio = 0.0;
  if (!(bb > 0.0)) {
    if ((e = cudaMemsetAsync(x, 0, sizeof(double) * V, s))) return e;
    k2m_report<<<1, 1, 0, s>>>(rec, 0, 0, 0.0, bb == 0.0 ? SGN_OK : SGN_ERR_BREAKDOWN);
    return cudaGetLastError();
  }
  const double bnorm = sqrt(bb);
  // r = b - G x
  auto residual = [&]() -> cudaError_t {
    cudaError_t r_ = applyG<double, double>(M, eta, gradh, x, q, l, s);
    if (r_) return r_;
    k2m_sub_scale<double><<<nb, 256, 0, s>>>(V, b, q, 1.0, r);
    return cudaGetLastError();
  };
  if (precision != SGN_PREC_MIXED) {
    double rz;
    if ((e = residual()) || (e = ainv<double, double>(M, rec, r, z, s)) ||
        (e = cudaMemcpyAsync(p, z, sizeof(double) * V, cudaMemcpyDeviceToDevice, s)) ||
        (e = dot_to(M, r, z, V, 0, s)) || (e = read_slots(M, 1, s)))
      return e;
    rz = H[0];
    const double tol = rtol * bnorm;
    while (sqrt(rz) > tol) {
      if (iters >= maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      if ((e = applyG<double, double>(M, eta, gradh, p, q, l, s)) ||
          (e = dot_to(M, p, q, V, 0, s)) || (e = read_slots(M, 1, s)))
        return e;
      const double pq = H[0];
      if (!(pq > 0.0) || !std::isfinite(pq)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double a = rz / pq;
      k2m_axpy<double><<<nb, 256, 0, s>>>(V, a, p, x);
      k2m_axpy<double><<<nb, 256, 0, s>>>(V, -a, q, r);
      if ((e = cudaGetLastError()) || (e = ainv<double, double>(M, rec, r, z, s)) ||
          (e = dot_to(M, r, z, V, 0, s)) || (e = read_slots(M, 1, s)))
        return e;
      const double rzn = H[0];
      ++iters;
      if (!std::isfinite(rzn)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double beta = rzn / rz;
      rz = rzn;
      k2m_xpby<double><<<nb, 256, 0, s>>>(V, z, beta, p);
      if ((e = cudaGetLastError())) return e;
    }
    ratio = sqrt(fmax(rz, 0.0)) / bnorm;
  } else {
    // float32 inner PCG for G d = r / ||r|| inside float64 refinement
    float* rf = M.fp(10);
    float* pf = M.fp(11);
    float* zf = M.fp(12);
    float* qf = M.fp(13);
    float* df_ = M.fp(14);
    float* lf = M.fp(15);
    const int cap = max_refine > 0 ? max_refine : 12;
    for (;;) {
      if ((e = residual()) || (e = ainv<double, double>(M, rec, r, z, s)) ||
          (e = dot_to(M, r, z, V, 0, s)) || (e = read_slots(M, 1, s)))
        return e;
      const double nr = sqrt(fmax(H[0], 0.0));
      ratio = nr / bnorm;
      if (ratio <= rtol) {
        status = SGN_OK;
        break;
      }
      if (status != SGN_OK) break;
      if (!std::isfinite(nr)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      if (refinements >= cap || iters >= maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      const double tin =
          rtol_inner > 0.0 ? rtol_inner : fmin(0.1, fmax(1e-6, 0.3 * rtol / ratio));
      k2m_scale_to<float><<<nb, 256, 0, s>>>(V, 1.0 / nr, r, rf);
      if ((e = cudaGetLastError()) ||
          (e = cudaMemsetAsync(df_, 0, sizeof(float) * V, s)) ||
          (e = ainv<float, float>(M, rec, rf, zf, s)) ||
          (e = cudaMemcpyAsync(pf, zf, sizeof(float) * V, cudaMemcpyDeviceToDevice, s)) ||
          (e = dot_to(M, rf, zf, V, 0, s)) || (e = read_slots(M, 1, s)))
        return e;
      double rzf = H[0];
      const int it0 = iters;
      int st_in = SGN_OK;
      while (sqrt(fmax(rzf, 0.0)) > tin) {
        if (iters >= maxit) {
          st_in = SGN_ERR_NOT_CONVERGED;
          break;
        }
        if ((e = applyG<float, float>(M, eta, gradh, pf, qf, lf, s)) ||
            (e = dot_to(M, pf, qf, V, 0, s)) || (e = read_slots(M, 1, s)))
          return e;
        const double pq = H[0];
        if (!(pq > 0.0) || !std::isfinite(pq)) {
          st_in = SGN_ERR_BREAKDOWN;
          break;
        }
        const double a = rzf / pq;
        k2m_axpy<float><<<nb, 256, 0, s>>>(V, a, pf, df_);
        k2m_axpy<float><<<nb, 256, 0, s>>>(V, -a, qf, rf);
        if ((e = cudaGetLastError()) || (e = ainv<float, float>(M, rec, rf, zf, s)) ||
            (e = dot_to(M, rf, zf, V, 0, s)) || (e = read_slots(M, 1, s)))
          return e;
        const double rzn = H[0];
        ++iters;
        if (!std::isfinite(rzn)) {
          st_in = SGN_ERR_BREAKDOWN;
          break;
        }
        const double beta = rzn / rzf;
        rzf = rzn;
        k2m_xpby<float><<<nb, 256, 0, s>>>(V, zf, beta, pf);
        if ((e = cudaGetLastError())) return e;
      }
      // a float32 breakdown after some progress keeps its correction (the next residual
      // decides); one without progress ends the solve
      if (st_in == SGN_ERR_BREAKDOWN && iters == it0) status = SGN_ERR_BREAKDOWN;
      k2m_correct<<<nb, 256, 0, s>>>(V, nr, df_, x);
      if ((e = cudaGetLastError())) return e;
      ++refinements;
    }
  }
  k2m_report<<<1, 1, 0, s>>>(rec, iters, refinements, ratio, status);
  return cudaGetLastError();
}

cudaError_t mr2d_rhs(const Layout2d& L, double g, const double* eta, const double* u,
                     const double* h, const double* gradh, double* f_eta, double* f_U,
                     cudaStream_t s) {
  const Mr M(L);
  const long long P = L.P;
  const int nb = blocks_for(P);
  double *sv = M.rp(0), *eu = M.rp(1), *ev = M.rp(2), *zeta = M.rp(3), *fu = M.rp(4),
         *fuv = M.rp(5), *fv = M.rp(6), *d = M.rp(7), *m = M.rp(8), *a1 = M.rp(9),
         *a2 = M.rp(10), *sx = M.rp(11), *sy = M.rp(12), *dx = M.rp(13), *dy = M.rp(14),
         *zx = M.rp(15), *zy = M.rp(16), *Phi = M.rp(17), *Psi = M.rp(18), *px = M.rp(19),
         *py = M.rp(20);
  k2m_rhs_pre<<<nb, 256, 0, s>>>(P, eta, u, h, gradh, sv, eu, ev, zeta, fu, fuv, fv);
  cudaError_t e = cudaGetLastError();
  if (!e) e = div2(M, u, u + P, d, s);             // d = div u
  if (!e) e = div2(M, eu, ev, m, s);               // m = div(eta u)
  if (!e) e = div2(M, fu, fuv, a1, s);             // div(eta u u^T), both components
  if (!e) e = div2(M, fuv, fv, a2, s);
  if (!e) e = grad2(M, sv, sx, sy, s);
  if (!e) e = grad2(M, d, dx, dy, s);
  if (!e) e = grad2(M, zeta, zx, zy, s);
  if (e) return e;
  k2m_rhs_mid<<<nb, 256, 0, s>>>(P, eta, u, d, m, sv, sx, sy, dx, dy, Phi, Psi);
  if ((e = cudaGetLastError()) || (e = grad2(M, Phi, px, py, s))) return e;
  k2m_rhs_end<<<nb, 256, 0, s>>>(P, g, eta, gradh, m, zx, zy, a1, a2, px, py, Psi, f_eta, f_U);
  return cudaGetLastError();
}

}  // namespace sgn
