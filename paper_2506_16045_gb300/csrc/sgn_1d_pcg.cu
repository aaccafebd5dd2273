// a5/a6: preconditioned conjugate gradients for G_{eta,h} x = b in 1d (§3.2, Eq:PCGLinSyst,
// preconditioner A of §4), one CTA per instance, in spectral space (see sgn_1d.cu).
//
//   MIXED = false: float64 PCG (TI = double) from the caller's initial guess.
//   MIXED = true : iterative refinement in double-float (~48-bit) precision.  Each pass
//                  computes the residual r = b - G x with double-float FFTs and
//                  coefficients, stops when sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b), and
//                  otherwise solves G d = r / ||r||_{A^{-1}} by float32 PCG (to rtol_inner,
//                  or adaptively to 0.3 rtol / current ratio within [1e-6, 0.1])
//                  and updates x += ||r||_{A^{-1}} d in double-float.  Float32 products are
//                  summed per thread (at most 2 MAXB + 1 terms) and the per-thread partials
//                  are summed across the CTA in float64.
//
// Workspace slots per instance (half spectra of n/2 + 1 modes, 16 bytes per mode each):
//   0: b^ (high precision), 1: x^ (high), 2: r^ (TI), 3: p^ (TI), 4: d^ (TI, mixed only),
//   5: G p (TI) inside PCG, and the high-precision residual between refinement passes.
// The mixed path also keeps the remainders of its double-float coefficients in coef_lo
// (3 floats per point).
#include <type_traits>

#include "sgn_1d_dev.cuh"

namespace sgn {
namespace {

using namespace d1;

template <typename T>
struct GetGlobal {
  const cplx<T>* p;
  __device__ __forceinline__ cplx<T> operator()(int m) const { return p[m]; }
};

// PCG on half-spectrum vectors: Rt holds the right-hand side residual on entry, Xt
// accumulates the iterate.  Stops when sqrt(r.A^{-1}r) <= tol_abs or after it_cap total
// iterations (counted in `iters`).  Returns the final r.A^{-1}r.  All per-mode work is in
// TT; only the CTA-wide sums are float64.
template <typename TT, int NT, int MAXB, typename Coef>
__device__ __forceinline__ double pcg_loop(cplx<TT>* fbuf, double* red, const Spec<TT>& sp,
                                           int log2n, cplx<TT>* __restrict__ Rt,
                                           cplx<TT>* __restrict__ Pt, cplx<TT>* __restrict__ Xt,
                                           cplx<TT>* __restrict__ Gt, const Coef& coef,
                                           const cplx<TT>* __restrict__ tw, double tol_abs,
                                           int it_cap, int& iters, int& status) {
  constexpr int MPT = 2 * MAXB + 1;
  const int n = sp.n, h = sp.h;
  double rz;
  {
    TT loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        TT k = sp.k(m);
        TT di = recip(sp.sigma + sp.alpha * k * k);
        cplx<TT> r = Rt[m];
        cplx<TT> z = r * di;
        Pt[m] = z;
        loc += sp.weight(m) * (r.x * z.x + r.y * z.y);
      }
    }
    rz = block_sum<NT>((double)loc, red);
  }
  while (sqrt(rz) > tol_abs) {
    if (iters >= it_cap) {
      status = SGN_ERR_NOT_CONVERGED;
      break;
    }
    spectral_matvec<TT, NT, MAXB>(fbuf, sp, log2n, GetGlobal<TT>{Pt}, coef, nullptr, tw);
    TT pq_loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        cplx<TT> g = gv_mode(fbuf, m, n, sp.k(m));
        Gt[m] = g;
        cplx<TT> p = Pt[m];
        pq_loc += sp.weight(m) * (p.x * g.x + p.y * g.y);
      }
    }
    const double pq = block_sum<NT>((double)pq_loc, red);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = SGN_ERR_BREAKDOWN;
      break;
    }
    const TT at = (TT)(rz / pq);
    TT rz_loc = 0;
#pragma unroll
    for (int b = 0; b < MPT; ++b) {
      int m = threadIdx.x + b * NT;
      if (m <= h) {
        TT k = sp.k(m);
        TT di = recip(sp.sigma + sp.alpha * k * k);
        cplx<TT> p = Pt[m];
        Xt[m] = Xt[m] + p * at;
        cplx<TT> r = Rt[m] - Gt[m] * at;
        Rt[m] = r;
        cplx<TT> z = r * di;
        rz_loc += sp.weight(m) * (r.x * z.x + r.y * z.y);
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
        TT k = sp.k(m);
        TT di = recip(sp.sigma + sp.alpha * k * k);
        Pt[m] = Rt[m] * di + Pt[m] * beta;
      }
    }
  }
  return rz;
}

// Float32 PCG with r^, p^ and G p held in registers (thread t owns modes t + b NT < n/2;
// thread 0 also owns the Nyquist mode n/2, whose wavenumber is 0).  R0 holds the
// right-hand side, Xt accumulates the iterate in global memory.  Same iteration and
// stopping rule as pcg_loop.  Dot products reduce in double-float across the CTA and
// thread 0 alone forms alpha, beta and the stopping decision, published through `sc`.
struct PcgScalars {
  double rz;      // current r.A^{-1}r
  float alpha, beta;
  int state;      // 0 iterate, 1 converged, 2 breakdown, 3 iteration cap
};

template <int NT, int MAXB>
__device__ __forceinline__ double pcg_loop_f32(cplx<float>* fbuf, df* slots, PcgScalars* sc,
                                               const Spec<float>& sp, int log2n,
                                               const cplx<float>* __restrict__ R0,
                                               cplx<float>* __restrict__ Xt,
                                               const CoefSmem32& coef, double tol_abs,
                                               int it_cap, int& iters, int& status) {
  constexpr int M = 2 * MAXB;
  constexpr int W = NT / 32;
  const int n = sp.n, h = sp.h, t = threadIdx.x;
  const bool nyq = (t == 0);
  const float dN = recip(sp.sigma);              // Nyquist: k = 0
  cplx<float> r[M], p[M], rN = mk(0.0f, 0.0f), pN = mk(0.0f, 0.0f);
  int it = iters;
  {
    float loc = 0.0f;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int m = t + b * NT;
      if (m < h) {
        const float k = sp.k(m);
        const float di = recip(sp.sigma + sp.alpha * k * k);
        r[b] = R0[m];
        p[b] = r[b] * di;
        loc += sp.weight(m) * (r[b].x * p[b].x + r[b].y * p[b].y);
      }
    }
    if (nyq) {
      rN = R0[h];
      pN = rN * dN;
      loc += rN.x * pN.x + rN.y * pN.y;
    }
    block_sum_df<NT>(loc, slots, [&](float hi, float lo) {
      const double rz = (double)hi + (double)lo;
      sc->rz = rz;
      sc->state = (sqrt(rz) <= tol_abs) ? 1 : (it >= it_cap ? 3 : 0);
    });
  }
  for (;;) {
    const int state = sc->state;
    if (state != 0) {
      if (state == 3) status = SGN_ERR_NOT_CONVERGED;
      if (state == 2) status = SGN_ERR_BREAKDOWN;
      break;
    }
    // Z = (1 - k) p for m < n/2, its conjugate mirror, and the Nyquist entry
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int m = t + b * NT;
      if (m < h) {
        const float k = sp.k(m);
        if (m > 0) {
          fbuf[m] = p[b] * (1.0f - k);
          fbuf[n - m] = conj(p[b]) * (1.0f + k);
        } else {
          fbuf[0] = mk(p[b].x, 0.0f);            // real DC coefficient
        }
      }
    }
    if (nyq) fbuf[h] = mk(pN.x, 0.0f);            // real Nyquist coefficient
    __syncthreads();
    matvec_core<float, NT, MAXB>(fbuf, n, log2n, coef, nullptr, nullptr);
    cplx<float> g[M], gN = mk(0.0f, 0.0f);
    float pq_loc = 0.0f;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int m = t + b * NT;
      if (m < h) {
        g[b] = gv_mode(fbuf, m, n, sp.k(m));
        pq_loc += sp.weight(m) * (p[b].x * g[b].x + p[b].y * g[b].y);
      }
    }
    if (nyq) {
      gN = gv_mode(fbuf, h, n, 0.0f);
      pq_loc += pN.x * gN.x + pN.y * gN.y;
    }
    block_sum_df<NT>(pq_loc, slots, [&](float hi, float lo) {
      const double pq = (double)hi + (double)lo;
      if (!(pq > 0.0) || !isfinite(pq)) {
        sc->state = 2;
      } else {
        sc->alpha = (float)(sc->rz / pq);
      }
    });
    if (sc->state == 2) {
      status = SGN_ERR_BREAKDOWN;
      break;
    }
    const float at = sc->alpha;
    float rz_loc = 0.0f;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int m = t + b * NT;
      if (m < h) {
        const float k = sp.k(m);
        const float di = recip(sp.sigma + sp.alpha * k * k);
        Xt[m] = Xt[m] + p[b] * at;
        r[b] = r[b] - g[b] * at;
        rz_loc += sp.weight(m) * (r[b].x * r[b].x + r[b].y * r[b].y) * di;
      }
    }
    if (nyq) {
      Xt[h] = Xt[h] + pN * at;
      rN = rN - gN * at;
      rz_loc += (rN.x * rN.x + rN.y * rN.y) * dN;
    }
    ++it;
    block_sum_df<NT>(rz_loc, slots + W, [&](float hi, float lo) {
      const double rz_new = (double)hi + (double)lo;
      if (!isfinite(rz_new)) {
        sc->state = 2;
      } else {
        sc->beta = (float)(rz_new / sc->rz);
        sc->rz = rz_new;
        sc->state = (sqrt(rz_new) <= tol_abs) ? 1 : (it >= it_cap ? 3 : 0);
      }
    });
    if (sc->state == 2) {
      status = SGN_ERR_BREAKDOWN;
      break;
    }
    const float beta = sc->beta;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const int m = t + b * NT;
      if (m < h) {
        const float k = sp.k(m);
        const float di = recip(sp.sigma + sp.alpha * k * k);
        p[b] = r[b] * di + p[b] * beta;
      }
    }
    if (nyq) pN = rN * dN + pN * beta;
  }
  iters = it;
  return sc->rz;
}

template <typename TI, int NT, int MAXB, bool MIXED>
__global__ void __launch_bounds__(NT, 1) k_pcg1d(const Inst1d* __restrict__ insts,
                                              const int* __restrict__ ids,
                                              const cplx<double>* __restrict__ tw64,
                                              const cplx<float>* __restrict__ tw32,
                                              const cplx<df>* __restrict__ twdf,
                                              const double* __restrict__ eta_all,
                                              const double* __restrict__ hx_all,
                                              const double* __restrict__ b_all,
                                              double* __restrict__ x_all,
                                              const SolveRec* __restrict__ given, int kind,
                                              double rtol, double rtol_inner, int maxit,
                                              int max_refine, SolveRec* __restrict__ rec,
                                              cplx<double>* __restrict__ ws,
                                              float* __restrict__ coef_lo_all) {
  using TH = typename std::conditional<MIXED, df, double>::type;   // high precision
  constexpr int MPT = 2 * MAXB + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[NT / 32 + 1];
  __shared__ df slots[2 * (NT / 32)];
  __shared__ PcgScalars sc;
  cplx<TH>* bufh = reinterpret_cast<cplx<TH>*>(smem);
  const cplx<TH>* twh;
  if constexpr (MIXED) twh = twdf; else twh = tw64;

  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1, log2n = I.log2n;
  const double* eta = eta_all + I.off;
  const double* hx = hx_all + I.off;
  const double* b = b_all + I.off;
  double* x = x_all + I.off;
  const long long S = h + 1;
  cplx<TH>* Bh = reinterpret_cast<cplx<TH>*>(ws + I.ws);
  cplx<TH>* Xh = reinterpret_cast<cplx<TH>*>(ws + I.ws + S);
  cplx<TI>* Rh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 2 * S);
  cplx<TI>* Ph = reinterpret_cast<cplx<TI>*>(ws + I.ws + 3 * S);
  cplx<TI>* Dh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 4 * S);
  cplx<TI>* Gh = reinterpret_cast<cplx<TI>*>(ws + I.ws + 5 * S);
  cplx<TH>* Wh = reinterpret_cast<cplx<TH>*>(ws + I.ws + 5 * S);

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
  const Spec<TH> sph = make_spec<TH>(n, I.L, R.sigma, R.alpha);
  const Spec<TI> spi = make_spec<TI>(n, I.L, R.sigma, R.alpha);

  float* c32 = reinterpret_cast<float*>(smem + (size_t)16 * n);
  float* clo = coef_lo_all ? coef_lo_all + 3 * I.off : nullptr;
  if constexpr (MIXED) split_coefficients<NT>(eta, hx, n, c32, clo);

  // ---- b^ and x0^ from one packed transform of b + i x0
  for (int j = threadIdx.x; j < n; j += NT) bufh[j] = mk(num<TH>(b[j]), num<TH>(x[j]));
  __syncthreads();
  cta_fft<TH, NT, MAXB>(bufh, n, log2n, false, twh);
  float bb_loc = 0.0f;
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<TH> z = bufh[m], zc = conj(bufh[(n - m) & (n - 1)]);
    cplx<TH> s = z + zc, d = mul_mi(z - zc);
    cplx<TH> bh = mk(half(s.x), half(s.y));
    Bh[m] = bh;
    Xh[m] = mk(half(d.x), half(d.y));
    float k = (float)spi.k(m);
    float bx = (float)to_f64(bh.x), by = (float)to_f64(bh.y);
    bb_loc += (float)spi.weight(m) * (bx * bx + by * by) /
              ((float)spi.sigma + (float)spi.alpha * k * k);
  }
  const double bb = block_sum<NT>((double)bb_loc, red);
  const double bnorm = sqrt(bb);
  if (!(bnorm > 0.0)) {
    for (int j = threadIdx.x; j < n; j += NT) x[j] = 0.0;
    R.status = (bb == 0.0) ? SGN_OK : SGN_ERR_BREAKDOWN;
    if (threadIdx.x == 0) rec[id] = R;
    return;
  }

  int iters = 0;
  int status = SGN_OK;
  if constexpr (!MIXED) {
    const CoefGlobal64 coef64{eta, hx};
    // r = b - G x0, then PCG on the whole system in float64
    spectral_matvec<double, NT, MAXB>(bufh, sph, log2n, GetGlobal<double>{Xh}, coef64, nullptr,
                                      tw64);
    for (int m = threadIdx.x; m <= h; m += NT) Rh[m] = Bh[m] - gv_mode(bufh, m, n, sph.k(m));
    __syncthreads();
    const double rz = pcg_loop<double, NT, MAXB>(bufh, red, sph, log2n, Rh, Ph, Xh, Gh, coef64,
                                                 tw64, rtol * bnorm, maxit, iters, status);
    R.ratio = sqrt(rz) / bnorm;
    for (int m = threadIdx.x; m <= h; m += NT) {
      cplx<double> v = Xh[m];
      bufh[m] = v;
      if (m > 0 && m < h) bufh[n - m] = conj(v);
    }
    __syncthreads();
    cta_fft<double, NT, MAXB>(bufh, n, log2n, true, tw64);
    const double inv_n = 1.0 / n;
    for (int j = threadIdx.x; j < n; j += NT) x[j] = bufh[j].x * inv_n;
  } else {
    cplx<float>* buf32 = reinterpret_cast<cplx<float>*>(smem);
    const CoefSmem32 coef32{c32, n};
    const CoefDF coefdf{c32, clo, n};
    int refinements = 0;
    for (;;) {
      // double-float residual r^ = b^ - (G x)^, writing the real-space x on the way
      spectral_matvec<df, NT, MAXB>(bufh, sph, log2n, GetGlobal<df>{Xh}, coefdf, x, twdf);
      float rz_loc = 0.0f;
#pragma unroll
      for (int bI = 0; bI < MPT; ++bI) {
        int m = threadIdx.x + bI * NT;
        if (m <= h) {
          cplx<df> rr = Bh[m] - gv_mode(bufh, m, n, sph.k(m));
          Wh[m] = rr;
          float k = spi.k(m);
          float di = recip(spi.sigma + spi.alpha * k * k);
          rz_loc += spi.weight(m) * (rr.x.hi * rr.x.hi + rr.y.hi * rr.y.hi) * di;
        }
      }
      const double rz64 = block_sum<NT>((double)rz_loc, red);
      R.ratio = sqrt(rz64) / bnorm;
      if (R.ratio <= rtol) break;
      if (status != SGN_OK) break;
      if (refinements >= max_refine || iters >= maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      const float scale = (float)(1.0 / sqrt(rz64));
#pragma unroll
      for (int bI = 0; bI < MPT; ++bI) {
        int m = threadIdx.x + bI * NT;
        if (m <= h) {
          cplx<df> rr = Wh[m];
          Rh[m] = mk((rr.x.hi + rr.x.lo) * scale, (rr.y.hi + rr.y.lo) * scale);
          Dh[m] = mk(0.0f, 0.0f);
        }
      }
      __syncthreads();
      int st_in = SGN_OK;
      // inner target: the reduction still needed (with a 0.3 margin), within what float32
      // PCG resolves, unless the caller fixed rtol_inner
      const double tin =
          rtol_inner > 0.0 ? rtol_inner : fmin(0.1, fmax(1e-6, 0.3 * rtol / R.ratio));
      const int it_before = iters;
      pcg_loop_f32<NT, MAXB>(buf32, slots, &sc, spi, log2n, Rh, Dh, coef32, tin, maxit, iters,
                             st_in);
      // A float32 breakdown after some progress only means float32 has resolved what it
      // can: keep the correction and let the next refinement pass decide.
      if (st_in == SGN_ERR_BREAKDOWN && iters == it_before) status = SGN_ERR_BREAKDOWN;
      ++refinements;
      const df unscale(sqrt(rz64));
      for (int m = threadIdx.x; m <= h; m += NT) {
        cplx<float> d = Dh[m];
        cplx<df> xv = Xh[m];
        Xh[m] = mk(xv.x + df(d.x, 0.0f) * unscale, xv.y + df(d.y, 0.0f) * unscale);
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
                         int maxit, int max_refine, SolveRec* rec, void* ws, float* coef_lo,
                         cudaStream_t s) {
  auto t64 = static_cast<const cplx<double>*>(tw64);
  auto t32 = static_cast<const cplx<float>*>(tw32);
  auto tdf = reinterpret_cast<const cplx<df>*>(static_cast<const char*>(tw32) + kTw32Bytes);
  auto w = static_cast<cplx<double>*>(ws);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    if (precision == SGN_PREC_MIXED) {
      size_t sm = ((size_t)16 << l) + ((size_t)12 << l);
      auto k = k_pcg1d<float, NT, MB, true>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, t64, t32, tdf, eta, hx, b, x, given,
                            kind, rtol, rtol_inner, maxit, max_refine, rec, w, coef_lo);
    } else {
      size_t sm = (size_t)16 << l;
      auto k = k_pcg1d<double, NT, MB, false>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, t64, t32, tdf, eta, hx, b, x, given,
                            kind, rtol, rtol_inner, maxit, max_refine, rec, w, nullptr);
    }
    return cudaGetLastError();
  });
}

}  // namespace sgn
