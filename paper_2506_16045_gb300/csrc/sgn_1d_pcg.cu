// a5/a6: preconditioned conjugate gradients for G_{eta,h} x = b in 1d (§3.2, Eq:PCGLinSyst,
// preconditioner A of §4), one CTA per instance, in spectral space (see sgn_1d.cu).
//
//   MIXED = false: float64 PCG (TI = double) from the caller's initial guess.
//   MIXED = true : float64 iterative refinement.  Each pass computes the float64 residual
//                  r = b - G x (float64 FFTs) and, unless sqrt(r.A^{-1}r) <= rtol
//                  sqrt(b.A^{-1}b), solves G d = r / ||r||_{A^{-1}} by float32 PCG to
//                  rtol_inner and updates x += ||r||_{A^{-1}} d in float64.  Float32
//                  products are summed per thread (at most 2 MAXB + 1 terms) and the
//                  per-thread partials are summed across the CTA in float64.
//
// Workspace slots per instance (half spectra of n/2 + 1 modes):
//   0: b^ (float64), 1: x^ (float64), 2: r^ (TI), 3: p^ (TI), 4: d^ (TI, mixed only),
//   5: G p (TI) inside PCG, and the float64 residual between refinement passes.
#include "sgn_1d_dev.cuh"

namespace sgn {
namespace {

using namespace d1;

template <typename T>
struct GetGlobal {
  const cplx<T>* p;
  __device__ __forceinline__ cplx<T> operator()(int m) const { return p[m]; }
};

__device__ __forceinline__ double mode_weight(int m, int h) { return (m == 0 || m == h) ? 1.0 : 2.0; }

// PCG on half-spectrum vectors: Rt holds the right-hand side residual on entry, Xt
// accumulates the iterate.  Stops when sqrt(r.A^{-1}r) <= tol_abs or after it_cap total
// iterations (counted in `iters`).  Returns the final r.A^{-1}r.
template <typename TT, int NT, int MAXB, typename Coef>
__device__ __forceinline__ double pcg_loop(cplx<TT>* fbuf, double* red, int n, int log2n,
                                           double kunit, double sigma, double alpha,
                                           cplx<TT>* __restrict__ Rt, cplx<TT>* __restrict__ Pt,
                                           cplx<TT>* __restrict__ Xt,
                                           cplx<TT>* __restrict__ Gt, const Coef& coef,
                                           const cplx<TT>* __restrict__ tw, double tol_abs,
                                           int it_cap, int& iters, int& status) {
  constexpr int MPT = 2 * MAXB + 1;
  const int h = n >> 1;
  double rz = 0.0;
  {
    TT loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        double k = mode_k(m, n, kunit);
        cplx<TT> r = Rt[m];
        cplx<TT> z = r * (TT)(1.0 / (sigma + alpha * k * k));
        Pt[m] = z;
        loc += (TT)mode_weight(m, h) * (r.x * z.x + r.y * z.y);
      }
    }
    rz = block_sum<NT>((double)loc, red);
  }
  while (sqrt(rz) > tol_abs) {
    if (iters >= it_cap) {
      status = SGN_ERR_NOT_CONVERGED;
      break;
    }
    spectral_matvec<TT, NT, MAXB>(fbuf, n, log2n, kunit, GetGlobal<TT>{Pt}, coef, nullptr, tw);
    TT pq_loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        cplx<TT> g = gv_mode(fbuf, m, n, (TT)mode_k(m, n, kunit));
        Gt[m] = g;
        cplx<TT> p = Pt[m];
        pq_loc += (TT)mode_weight(m, h) * (p.x * g.x + p.y * g.y);
      }
    }
    const double pq = block_sum<NT>((double)pq_loc, red);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = SGN_ERR_BREAKDOWN;
      break;
    }
    const double a = rz / pq;
    const TT at = (TT)a;
    TT rz_loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        double k = mode_k(m, n, kunit);
        cplx<TT> p = Pt[m];
        Xt[m] = Xt[m] + p * at;
        cplx<TT> r = Rt[m] - Gt[m] * at;
        Rt[m] = r;
        cplx<TT> z = r * (TT)(1.0 / (sigma + alpha * k * k));
        rz_loc += (TT)mode_weight(m, h) * (r.x * z.x + r.y * z.y);
      }
    }
    const double rz_new = block_sum<NT>((double)rz_loc, red);
    ++iters;
    if (!isfinite(rz_new)) {
      status = SGN_ERR_BREAKDOWN;
      break;
    }
    const TT beta = (TT)(rz_new / rz);
    rz = rz_new;
    // p = z + beta p with z = A^{-1} r recomputed from the r each thread just wrote
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        double k = mode_k(m, n, kunit);
        Pt[m] = Rt[m] * (TT)(1.0 / (sigma + alpha * k * k)) + Pt[m] * beta;
      }
    }
  }
  return rz;
}

template <typename TI, int NT, int MAXB, bool MIXED>
__global__ void __launch_bounds__(NT) k_pcg1d(const Inst1d* __restrict__ insts,
                                              const int* __restrict__ ids,
                                              const cplx<double>* __restrict__ tw64,
                                              const cplx<float>* __restrict__ tw32,
                                              const double* __restrict__ eta_all,
                                              const double* __restrict__ hx_all,
                                              const double* __restrict__ b_all,
                                              double* __restrict__ x_all,
                                              const SolveRec* __restrict__ given, int kind,
                                              double rtol, double rtol_inner, int maxit,
                                              int max_refine, SolveRec* __restrict__ rec,
                                              cplx<double>* __restrict__ ws) {
  constexpr int MPT = 2 * MAXB + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[NT / 32 + 1];
  cplx<double>* buf64 = reinterpret_cast<cplx<double>*>(smem);

  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1, log2n = I.log2n;
  const double kunit = 2.0 * kPi / I.L;
  const double* eta = eta_all + I.off;
  const double* hx = hx_all + I.off;
  const double* b = b_all + I.off;
  double* x = x_all + I.off;
  const long long S = h + 1;
  cplx<double>* Bh = ws + I.ws;
  cplx<double>* Xh = ws + I.ws + S;
  cplx<TI>* Rh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 2 * S);
  cplx<TI>* Ph = reinterpret_cast<cplx<TI>*>(ws + I.ws + 3 * S);
  cplx<TI>* Dh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 4 * S);
  cplx<TI>* Gh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 5 * S);     // G p (TI)
  cplx<double>* Wh = ws + I.ws + 5 * S;                                 // float64 residual

  // ---- a1: coefficients (or the caller's)
  SolveRec R = {};
  if (given) {
    R = given[id];
    R.status = SGN_OK;
  } else {
    coeffs_block<NT>(eta, hx, n, kind, red, R);
  }
  R.iters = 0;
  R.refinements = 0;
  R.ratio = 0.0;
  if (R.status != SGN_OK) {
    if (threadIdx.x == 0) rec[id] = R;
    return;
  }
  const double sigma = R.sigma, alpha = R.alpha;

  float* c32 = reinterpret_cast<float*>(smem + (size_t)16 * n);
  if constexpr (MIXED) {
    for (int j = threadIdx.x; j < n; j += NT) {
      double e = eta[j], g = hx[j];
      c32[j] = (float)(e * (1.0 + g * g));
      c32[n + j] = (float)(0.5 * e * e * g);
      c32[2 * n + j] = (float)(e * e * e * (1.0 / 3.0));
    }
  }

  // ---- b^ and x0^ from one packed transform of b + i x0
  for (int j = threadIdx.x; j < n; j += NT) buf64[j] = mk(b[j], x[j]);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf64, n, log2n, false, tw64);
  double bb = 0.0;
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<double> z = buf64[m], zc = conj(buf64[(n - m) & (n - 1)]);
    cplx<double> bh = (z + zc) * 0.5;
    Bh[m] = bh;
    Xh[m] = mul_mi(z - zc) * 0.5;
    double k = mode_k(m, n, kunit);
    bb += mode_weight(m, h) * (bh.x * bh.x + bh.y * bh.y) / (sigma + alpha * k * k);
  }
  bb = block_sum<NT>(bb, red);
  const double bnorm = sqrt(bb);
  if (!(bnorm > 0.0)) {
    for (int j = threadIdx.x; j < n; j += NT) x[j] = 0.0;
    R.status = (bb == 0.0) ? SGN_OK : SGN_ERR_BREAKDOWN;
    if (threadIdx.x == 0) rec[id] = R;
    return;
  }

  const CoefGlobal64 coef64{eta, hx};
  int iters = 0;
  int status = SGN_OK;
  if constexpr (!MIXED) {
    // r = b - G x0, then PCG on the whole system in float64
    spectral_matvec<double, NT, MAXB>(buf64, n, log2n, kunit, GetGlobal<double>{Xh}, coef64,
                                      nullptr, tw64);
    for (int m = threadIdx.x; m <= h; m += NT)
      Rh[m] = Bh[m] - gv_mode(buf64, m, n, mode_k(m, n, kunit));
    __syncthreads();
    const double rz = pcg_loop<double, NT, MAXB>(buf64, red, n, log2n, kunit, sigma, alpha, Rh, Ph,
                                                 Xh, Gh, coef64, tw64, rtol * bnorm, maxit, iters,
                                                 status);
    R.ratio = sqrt(rz) / bnorm;
    for (int m = threadIdx.x; m <= h; m += NT) {
      cplx<double> v = Xh[m];
      buf64[m] = v;
      if (m > 0 && m < h) buf64[n - m] = conj(v);
    }
    __syncthreads();
    cta_fft<double, NT, MAXB>(buf64, n, log2n, true, tw64);
    const double inv_n = 1.0 / n;
    for (int j = threadIdx.x; j < n; j += NT) x[j] = buf64[j].x * inv_n;
  } else {
    cplx<float>* buf32 = reinterpret_cast<cplx<float>*>(smem);
    const CoefSmem32 coef32{c32, n};
    int refinements = 0;
    for (;;) {
      // float64 residual r^ = b^ - (G x)^, writing the real-space x on the way
      spectral_matvec<double, NT, MAXB>(buf64, n, log2n, kunit, GetGlobal<double>{Xh}, coef64, x,
                                        tw64);
      double rz64 = 0.0;
#pragma unroll
      for (int bI = 0; bI < MPT; ++bI) {
        int m = threadIdx.x + bI * NT;
        if (m <= h) {
          double k = mode_k(m, n, kunit);
          cplx<double> rr = Bh[m] - gv_mode(buf64, m, n, k);
          Wh[m] = rr;
          rz64 += mode_weight(m, h) * (rr.x * rr.x + rr.y * rr.y) / (sigma + alpha * k * k);
        }
      }
      rz64 = block_sum<NT>(rz64, red);
      R.ratio = sqrt(rz64) / bnorm;
      if (R.ratio <= rtol) break;
      if (status != SGN_OK) break;
      if (refinements >= max_refine || iters >= maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      const double scale = 1.0 / sqrt(rz64);
#pragma unroll
      for (int bI = 0; bI < MPT; ++bI) {
        int m = threadIdx.x + bI * NT;
        if (m <= h) {
          cplx<double> rr = Wh[m];
          Rh[m] = mk((float)(rr.x * scale), (float)(rr.y * scale));
          Dh[m] = mk(0.0f, 0.0f);
        }
      }
      int st_in = SGN_OK;
      pcg_loop<float, NT, MAXB>(buf32, red, n, log2n, kunit, sigma, alpha, Rh, Ph, Dh, Gh, coef32,
                                tw32, rtol_inner, maxit, iters, st_in);
      if (st_in == SGN_ERR_BREAKDOWN) status = SGN_ERR_BREAKDOWN;
      ++refinements;
      const double unscale = sqrt(rz64);
      for (int m = threadIdx.x; m <= h; m += NT) {
        cplx<float> d = Dh[m];
        cplx<double> xv = Xh[m];
        Xh[m] = mk(xv.x + (double)d.x * unscale, xv.y + (double)d.y * unscale);
      }
      __syncthreads();
    }
    R.refinements = refinements;
  }
  R.iters = iters;
  R.status = status;
  if (threadIdx.x == 0) rec[id] = R;
}

}  // namespace

cudaError_t launch_pcg1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         const double* eta, const double* hx, const double* b, double* x,
                         const SolveRec* given, int kind, double rtol, double rtol_inner,
                         int maxit, int max_refine, SolveRec* rec, void* ws, cudaStream_t s) {
  auto t64 = static_cast<const cplx<double>*>(tw64);
  auto t32 = static_cast<const cplx<float>*>(tw32);
  auto w = static_cast<cplx<double>*>(ws);
  return for_each_class(lay, [&](auto NTc, auto MBc, int l, int first, int num) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    if (precision == SGN_PREC_MIXED) {
      size_t sm = ((size_t)16 << l) + ((size_t)12 << l);
      auto k = k_pcg1d<float, NT, MB, true>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, t64, t32, eta, hx, b, x, given, kind,
                            rtol, rtol_inner, maxit, max_refine, rec, w);
    } else {
      size_t sm = (size_t)16 << l;
      auto k = k_pcg1d<double, NT, MB, false>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, t64, t32, eta, hx, b, x, given, kind,
                            rtol, rtol_inner, maxit, max_refine, rec, w);
    }
    return cudaGetLastError();
  });
}

}  // namespace sgn
