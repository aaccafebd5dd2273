// a7: right-hand side of Eq:DAE_DSWE with F from Def:bigF, one CTA per 1d instance on the
// register-blocked FFT of sgn_fft1d.cuh, in number type T (float64 for the float64 path,
// double-float for the mixed path).  Four derivative pairs:
//   (u, eta u) -> (d, m);  (zeta, s) -> (zeta_x, s_x) with s = h_x u;  d -> d_x;
//   Phi' -> Phi'_x with Phi' = eta^3 Q/3 + eta^2 m d + eta^2 S/2 + eta m s - eta u^2 (the
//   flux -(eta u^2)_x folded in), Q = u d_x - d^2, S = u s_x (reading R6);
// and f_eta = -m, f_U = -g eta zeta_x + Phi'_x - h_x Psi, Psi = eta^2 Q/2 + eta m d + eta S
// + m s.  Every pointwise step works on the thread's natural elements j = t + e NTA, so the
// intermediate planes in `scratch` are written and read by the same thread.  n = 16384 runs
// on a cluster of two CTAs, each holding half of the points (sgn_fft1d.cuh's two-CTA
// transforms).
#pragma once
#include <type_traits>

#include "sgn_1d_dev.cuh"
#include "sgn_fft1d.cuh"

namespace sgn {

struct RhsArgs {
  const Inst1d* insts;
  const int* ids;
  const cplx<double>* tw64;
  const cplx<df>* twdf;
  double g;
  const double* eta;
  const double* u;
  const double* h;
  const double* hx;
  double* f_eta;
  double* f_U;
  double* scratch;        // 5 planes of P values (8 bytes each)
  long long P;
  int precision;
  int ux_given;           // 1: the first scratch plane already holds u_x (see rhs_body)
};

// LG = log2 n; CL = CTAs per instance (2: thread-block clusters of two CTAs of the
// 2^(LG-1)-point kernel; the only form for LG = 14)
template <int LG, int CL>
cudaError_t rhs1d_launch(const RhsArgs& a, int first, int num, cudaStream_t s);

namespace rhs1d {

using namespace d1;
using f1::Plan;
using f1::XBuf;

// v <- D v for the two real fields packed in v (the thread's natural elements in and out):
// forward transform, i k_m / n on every mode (Nyquist 0), inverse transform as
// conj(F(conj .)).  Each thread touches only its own natural positions of X outside the
// transforms, so no barrier is needed around them.  CL = 2: X holds rank r's points and,
// after the split, its modes m = 2 k + r; XP is the partner's buffer.
template <typename T, int L, int CL>
__device__ __forceinline__ void deriv_pair(const XBuf<T>& X, const XBuf<T>& XP,
                                           cplx<T> (&v)[Plan<L>::E], int t, int bnat,
                                           bool act, unsigned rk, T kn,
                                           const cplx<T>* __restrict__ tw) {
  using PL = Plan<L>;
  if constexpr (CL > 1) {
    f1::cross<T, L, f1::kSplitFwd>(X, XP, v, t, bnat, act, rk, tw);
  }
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) X.st(bnat ^ f1::swz_c(e * PL::NTA), v[e]);
  }
  f1::fft_smem<T, L>(X, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) {
      const int a = bnat ^ f1::swz_c(e * PL::NTA);
      const int m = CL * (t + e * PL::NTA) + (int)rk;
      const T k = kn * from_int<T>(wave_index(m, CL * PL::n));
      X.st(a, conj(mul_pi(X.ld(a)) * k));
    }
  }
  f1::fft_smem<T, L>(X, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) v[e] = X.ld(bnat ^ f1::swz_c(e * PL::NTA));
  }
  if constexpr (CL > 1) {
    f1::cross<T, L, f1::kJoinConj>(X, XP, v, t, bnat, act, rk, tw);
  }
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) v[e] = conj(v[e]);
  }
}

// The right-hand side of one instance by one CTA.  UXG: d = u_x is already in the first
// scratch plane (written by the solve that produced u, in the same precision), so the
// derivative pairs are (eta u, zeta) -> (m, zeta_x), (s, d) -> (s_x, d_x) and Phi': six
// transforms instead of eight.
template <typename T, int L, bool UXG, int CL>
__device__ __forceinline__ void rhs_body(const RhsArgs& A, int first) {
  using PL = Plan<L>;
  constexpr int nl = PL::n, n = CL * nl, E = PL::E, NTA = PL::NTA;
  extern __shared__ __align__(16) unsigned char smem[];
  const int t = threadIdx.x;
  const unsigned rk = CL > 1 ? cluster_rank() : 0u;
  const Inst1d I = A.insts[A.ids[first + (CL > 1 ? (int)(blockIdx.x / CL) : (int)blockIdx.x)]];
  const long long own = I.off + (long long)rk * nl;    // first point of this CTA
  const T kn = num<T>(2.0 * kPi / I.L / (double)n);
  const T third = num<T>(1.0 / 3.0);
  const T gT = num<T>(A.g);
  const XBuf<T> X(smem, nl);
  const XBuf<T> XP = CL > 1 ? XBuf<T>(peer(smem), nl) : X;
  const cplx<T>* tw = std::is_same<T, df>::value ? reinterpret_cast<const cplx<T>*>(A.twdf)
                                                 : reinterpret_cast<const cplx<T>*>(A.tw64);
  const int bnat = f1::swz(t);
  const bool act = !PL::kIdle || t < NTA;
  const double* eta = A.eta + own;
  const double* u = A.u + own;
  const double* hh = A.h + own;
  const double* hx = A.hx + own;
  T* sd = reinterpret_cast<T*>(A.scratch + own);              // d = u_x
  T* sm = reinterpret_cast<T*>(A.scratch + A.P + own);        // m = (eta u)_x
  T* szx = reinterpret_cast<T*>(A.scratch + 2 * A.P + own);   // zeta_x
  T* ssx = reinterpret_cast<T*>(A.scratch + 3 * A.P + own);   // s_x
  T* spsi = reinterpret_cast<T*>(A.scratch + 4 * A.P + own);  // Psi
  cplx<T> v[E];
  if constexpr (UXG) {
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        const T ej = num<T>(eta[j]);
        v[e] = mk(ej * num<T>(u[j]), ej - num<T>(hh[j]));
      }
    }
    deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        sm[j] = v[e].x;
        szx[j] = v[e].y;
        v[e] = mk(num<T>(hx[j]) * num<T>(u[j]), sd[j]);
      }
    }
    deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);   // v = (s_x, d_x)
  } else {
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        const T uj = num<T>(u[j]);
        v[e] = mk(uj, num<T>(eta[j]) * uj);
      }
    }
    deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        sd[j] = v[e].x;
        sm[j] = v[e].y;
        v[e] = mk(num<T>(eta[j]) - num<T>(hh[j]), num<T>(hx[j]) * num<T>(u[j]));
      }
    }
    deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        szx[j] = v[e].x;
        ssx[j] = v[e].y;
        v[e] = mk(sd[j], from_int<T>(0));
      }
    }
    deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);   // v.x = d_x
  }
  if (act) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = t + e * NTA;
      const T ej = num<T>(eta[j]), uj = num<T>(u[j]), d = sd[j], m = sm[j];
      const T dx = UXG ? v[e].y : v[e].x;
      const T sx = UXG ? v[e].x : ssx[j];
      const T s = num<T>(hx[j]) * uj;
      const T Q = uj * dx - d * d;
      const T Sv = uj * sx;
      const T e2 = ej * ej;
      const T md = m * d;
      const T Phi = e2 * ej * Q * third + e2 * md + half(e2 * Sv) + ej * m * s - ej * uj * uj;
      spsi[j] = half(e2 * Q) + ej * md + ej * Sv + m * s;
      v[e] = mk(Phi, from_int<T>(0));
    }
  }
  deriv_pair<T, L, CL>(X, XP, v, t, bnat, act, rk, kn, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = t + e * NTA;
      A.f_eta[own + j] = -to_f64(sm[j]);
      const T fU = v[e].x - gT * num<T>(eta[j]) * szx[j] - num<T>(hx[j]) * spsi[j];
      A.f_U[own + j] = to_f64(fU);
    }
  }
}

template <typename T, int L, bool UXG, int CL>
__global__ void __launch_bounds__(Plan<L>::NT, Plan<L>::kMinBlocks)
    k_rhs1d(const __grid_constant__ RhsArgs A, int first) {
  rhs_body<T, L, UXG, CL>(A, first);
  // a CTA's shared memory must outlive the partner's last read of it
  if constexpr (CL > 1) cluster_sync();
}

}  // namespace rhs1d

template <int LG, int CL>
cudaError_t rhs1d_launch(const RhsArgs& a, int first, int num, cudaStream_t s) {
  static_assert(CL == 1 || CL == 2, "one CTA or a cluster of two per instance");
  static_assert(LG <= kSmemLog1d || CL == 2, "n = 16384 needs two CTAs");
  constexpr int L = LG - (CL - 1);          // points per CTA: 2^L
  using PL = f1::Plan<L>;
  const size_t sm = (size_t)16 << L;
  auto go = [&](auto k) -> cudaError_t {
    cudaError_t e = d1::set_smem(k, sm);
    if (e) return e;
    return d1::launch_clustered<CL>(k, num, PL::NT, sm, s, a, first);
  };
  if (a.precision == SGN_PREC_MIXED)
    return a.ux_given ? go(rhs1d::k_rhs1d<df, L, true, CL>) : go(rhs1d::k_rhs1d<df, L, false, CL>);
  return a.ux_given ? go(rhs1d::k_rhs1d<double, L, true, CL>)
                    : go(rhs1d::k_rhs1d<double, L, false, CL>);
}

}  // namespace sgn
