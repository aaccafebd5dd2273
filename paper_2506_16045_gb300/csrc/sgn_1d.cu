// 1d periodic SGN kernels: one CTA owns one instance and keeps the whole transform in
// shared memory (n <= 8192), so a PCG solve never leaves the SM between iterations.  The
// float64 helper kernels of this file (derivative, G apply, A solve, SBDF2 pieces) take the
// transform buffer of n = 16384 from a global scratch (`big`, L2-resident) instead; the
// solve and right-hand side run n = 16384 on two-CTA clusters (sgn_1d_pcg.cuh,
// sgn_1d_rhs.cuh).
//
// Spectral-space PCG.  All Krylov vectors live as half spectra (modes 0..n/2 of real
// fields).  One iteration needs two complex FFTs of length n:
//   * inverse FFT of Z_m = (1 - k_m) p_m gives n (p + i p_x) (the real field and its
//     derivative packed into one complex transform),
//   * pointwise w = c1 p + c2 p_x, q = c2 p + c3 p_x with c1 = eta (1 + h_x^2),
//     c2 = eta^2 h_x / 2, c3 = eta^3 / 3 (the 1d blocks of Def:MatrixM),
//   * forward FFT of w + i q = Y, and (G p)_m = w_m - i k_m q_m
//     = ((1 - k_m) Y_m + (1 + k_m) conj(Y_{n-m})) / 2, which is Def:G in 1d
//     (G p = w - (q)_x).
// Inner products use Parseval on half spectra (weight 1 for m = 0, n/2 and 2 otherwise);
// the common factor 1/n cancels in every ratio PCG forms.
#include <cstdio>
#include <type_traits>

#include "sgn_1d_dev.cuh"

namespace sgn {

namespace {

using namespace d1;

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------

__global__ void k_twiddles(cplx<double>* tw64, cplx<float>* tw32, cplx<df>* twdf) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kTwiddleN) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)kTwiddleN, &s, &c);
    tw64[j] = mk(c, s);
    tw32[j] = mk((float)c, (float)s);
    twdf[j] = mk(df(c), df(s));
  }
}

// f_x = D f, one field per CTA (complex transform with zero imaginary part)
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_deriv1d(const Inst1d* __restrict__ insts,
                                                const int* __restrict__ ids,
                                                cplx<double>* big,
                                                const cplx<double>* __restrict__ tw,
                                                const double* __restrict__ f,
                                                double* __restrict__ fx) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = big ? big + ((size_t)blockIdx.x << kMaxLog1d)
                          : reinterpret_cast<cplx<double>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n;
  const double kunit = 2.0 * kPi / I.L;
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(f[I.off + j], 0.0);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, false, tw);
  const double inv_n = 1.0 / n;
  for (int m = threadIdx.x; m < n; m += NT) {
    double k = kunit * (double)wave_index(m, n) * inv_n;
    buf[m] = mul_pi(buf[m]) * k;
  }
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, true, tw);
  for (int j = threadIdx.x; j < n; j += NT) fx[I.off + j] = buf[j].x;
}

// Gu (Def:G) in float64
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_apply_G1d(const Inst1d* __restrict__ insts,
                                                  const int* __restrict__ ids,
                                                  cplx<double>* big,
                                                  const cplx<double>* __restrict__ tw,
                                                  const double* __restrict__ eta,
                                                  const double* __restrict__ hx,
                                                  const double* __restrict__ u,
                                                  double* __restrict__ Gu) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = big ? big + ((size_t)blockIdx.x << kMaxLog1d)
                          : reinterpret_cast<cplx<double>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n, h = n >> 1;
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(u[I.off + j], 0.0);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, false, tw);
  CoefGlobal64 coef{eta + I.off, hx + I.off};
  const Spec<double> sp = make_spec<double>(n, I.L, 0.0, 0.0);
  spectral_matvec<double, NT, MAXB>(buf, sp, I.log2n, [&](int m) { return buf[m]; }, coef,
                                    nullptr, tw);
  // (G u)_m for m in [0, n/2]; the field is real, so (G u)_{n-m} = conj((G u)_m).
  cplx<double> g[2 * MAXB + 1];
#pragma unroll
  for (int b = 0; b < 2 * MAXB + 1; ++b) {
    int m = threadIdx.x + b * NT;
    if (m <= h) g[b] = gv_mode(buf, m, n, sp.k(m));
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < 2 * MAXB + 1; ++b) {
    int m = threadIdx.x + b * NT;
    if (m <= h) {
      buf[m] = g[b];
      if (m > 0 && m < h) buf[n - m] = conj(g[b]);
    }
  }
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, true, tw);
  const double inv_n = 1.0 / n;
  for (int j = threadIdx.x; j < n; j += NT) Gu[I.off + j] = buf[j].x * inv_n;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_coeffs1d(const Inst1d* __restrict__ insts,
                                                 const int* __restrict__ ids,
                                                 const double* __restrict__ eta,
                                                 const double* __restrict__ hx, int kind,
                                                 SolveRec* __restrict__ rec) {
  __shared__ double red[NT / 32 + 1];
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  SolveRec R = {};
  coeffs_block<NT>(eta + I.off, hx + I.off, I.n, kind, red, R);
  if (threadIdx.x == 0) rec[id] = R;
}

// z = A^{-1} r (Def:A): divide mode m by sigma + alpha k_m^2
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_precond1d(const Inst1d* __restrict__ insts,
                                                  const int* __restrict__ ids,
                                                  cplx<double>* big,
                                                  const cplx<double>* __restrict__ tw,
                                                  const SolveRec* __restrict__ rec,
                                                  const double* __restrict__ r,
                                                  double* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = big ? big + ((size_t)blockIdx.x << kMaxLog1d)
                          : reinterpret_cast<cplx<double>*>(smem);
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n;
  const double kunit = 2.0 * kPi / I.L;
  const double sigma = rec[id].sigma, alpha = rec[id].alpha;
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(r[I.off + j], 0.0);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, false, tw);
  for (int m = threadIdx.x; m < n; m += NT) {
    double k = kunit * (double)wave_index(m, n);
    buf[m] = buf[m] * (1.0 / ((sigma + alpha * k * k) * (double)n));
  }
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, true, tw);
  for (int j = threadIdx.x; j < n; j += NT) z[I.off + j] = buf[j].x;
}

struct AxpyArgs {
  const double* f[4];
  double c[4];
  int nterms;
};

// out = base + scale * dt_i * sum_t c_t f_t   (per-instance dt)
__global__ void k_axpy1d(const Inst1d* __restrict__ insts, const double* __restrict__ dt,
                         double* __restrict__ out, const double* __restrict__ base, AxpyArgs a,
                         double scale) {
  const Inst1d I = insts[blockIdx.x];
  const double s = scale * dt[blockIdx.x];
  for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
    const long long q = I.off + j;
    double acc = 0.0;
    for (int t = 0; t < a.nterms; ++t) acc += a.c[t] * a.f[t][q];
    out[q] = base[q] + s * acc;
  }
}

// Orszag's 2/3 rule on a new time level: the modes |j| > n/3 of zeta = eta - h, of U and
// (if u is non-null) of u are set to zero.  zeta and U share one complex transform
// (zeta + i U): the mask is symmetric in j and n - j, so masking the packed spectrum masks
// both fields exactly, and a projection does not amplify the shared rounding.  u takes a
// second transform.  Transforms in T: float64, or double-float on the mixed path.
template <typename T, int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_dealias1d(const Inst1d* __restrict__ insts,
                                                  const int* __restrict__ ids,
                                                  cplx<double>* big,
                                                  const cplx<T>* __restrict__ tw,
                                                  const double* __restrict__ h_all,
                                                  double* __restrict__ eta_all,
                                                  double* __restrict__ U_all,
                                                  double* __restrict__ u_all) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = big ? reinterpret_cast<cplx<T>*>(big + ((size_t)blockIdx.x << kMaxLog1d))
                     : reinterpret_cast<cplx<T>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n;
  const double inv_n = 1.0 / n, third = n / 3.0;
  const double* h = h_all + I.off;
  double* eta = eta_all + I.off;
  double* U = U_all + I.off;
  for (int pass = 0; pass < 2; ++pass) {
    double* f = pass == 0 ? eta : (u_all ? u_all + I.off : nullptr);
    if (!f) break;
    for (int j = threadIdx.x; j < n; j += NT)
      buf[j] = pass == 0 ? mk(num<T>(f[j] - h[j]), num<T>(U[j])) : mk(num<T>(f[j]), num<T>(0.0));
    __syncthreads();
    cta_fft<T, NT, MAXB>(buf, n, I.log2n, false, tw);
    for (int j = threadIdx.x; j < n; j += NT) {
      const int a = j <= n / 2 ? j : n - j;            // |wavenumber index|
      if (a > third) buf[j] = mk(num<T>(0.0), num<T>(0.0));
    }
    __syncthreads();
    cta_fft<T, NT, MAXB>(buf, n, I.log2n, true, tw);
    for (int j = threadIdx.x; j < n; j += NT) {
      if (pass == 0) {
        f[j] = to_f64(buf[j].x) * inv_n + h[j];
        U[j] = to_f64(buf[j].y) * inv_n;
      } else {
        f[j] = to_f64(buf[j].x) * inv_n;
      }
    }
    __syncthreads();                                    // buf is reused by the next pass
  }
}

// Right-hand side of the non-constraint form (Eq:dswe with the u_t terms grouped as in
// Eq:MomEq), per instance: f_eta = -(eta u)_x and
//   M = -eta u u_x - g eta zeta_x + (eta^3 Q/3 + eta^2 S/2)_x - h_x (eta^2 Q/2 + eta S),
//   Q = u u_xx - u_x^2, S = u (h_x u)_x,
// from three derivative pairs (u, h_x u), (u_x, zeta), (eta^3 Q/3 + eta^2 S/2, eta u) with
// transforms in T; the pointwise terms are formed in float64.  w0, w1: two packed real
// scratch fields.
template <typename T, int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_rhs_nc1d(const Inst1d* __restrict__ insts,
                                                 const int* __restrict__ ids, cplx<double>* big,
                                                 const cplx<T>* __restrict__ tw, double g,
                                                 const double* __restrict__ eta_all,
                                                 const double* __restrict__ u_all,
                                                 const double* __restrict__ h_all,
                                                 const double* __restrict__ hx_all,
                                                 double* __restrict__ fe_all,
                                                 double* __restrict__ M_all,
                                                 double* __restrict__ w0_all,
                                                 double* __restrict__ w1_all) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = big ? reinterpret_cast<cplx<T>*>(big + ((size_t)blockIdx.x << kMaxLog1d))
                     : reinterpret_cast<cplx<T>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n;
  const double* eta = eta_all + I.off;
  const double* u = u_all + I.off;
  const double* h = h_all + I.off;
  const double* hx = hx_all + I.off;
  double* fe = fe_all + I.off;
  double* M = M_all + I.off;
  double* w0 = w0_all + I.off;
  double* w1 = w1_all + I.off;
  const T ku = num<T>(2.0 * kPi / I.L / (double)n);
  // (u, h_x u) -> (d = u_x, s_x)
  deriv_pair<T, NT, MAXB>(buf, n, I.log2n, ku,
                          [&](int j) { return mk(num<T>(u[j]), num<T>(hx[j] * u[j])); }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    w0[j] = to_f64(buf[j].x);
    w1[j] = to_f64(buf[j].y);
  }
  __syncthreads();
  // (d, zeta) -> (d_x, zeta_x); the local terms of M, and Phi into w1
  deriv_pair<T, NT, MAXB>(buf, n, I.log2n, ku,
                          [&](int j) { return mk(num<T>(w0[j]), num<T>(eta[j] - h[j])); }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    const double e = eta[j], uj = u[j], d = w0[j], dx = to_f64(buf[j].x);
    const double zx = to_f64(buf[j].y);
    const double Q = uj * dx - d * d, S = uj * w1[j];
    M[j] = -e * uj * d - g * e * zx - hx[j] * (e * e * Q * 0.5 + e * S);
    w1[j] = e * e * e * Q * (1.0 / 3.0) + e * e * S * 0.5;
  }
  __syncthreads();
  // (Phi, eta u) -> (Phi_x, (eta u)_x)
  deriv_pair<T, NT, MAXB>(buf, n, I.log2n, ku,
                          [&](int j) { return mk(num<T>(w1[j]), num<T>(eta[j] * u[j])); }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    M[j] += to_f64(buf[j].x);
    fe[j] = -to_f64(buf[j].y);
  }
}

// double-float coefficients of Def:MatrixM computed from float64 eta and h_x on the fly
// (the products in double-float arithmetic, on the float32 units: only eta and h_x are
// split from float64)
struct CoefGlobalDF {
  const double* eta;
  const double* hx;
  __device__ __forceinline__ void operator()(int j, df& c1, df& c2, df& c3) const {
    const df e(eta[j]), g(hx[j]);
    const df e2 = e * e;
    c1 = e + e * (g * g);
    c2 = half(e2 * g);
    c3 = e2 * e * df(0.3333333432674408f, -9.934107758624577e-09f);   // 1/3, double-float
  }
};

template <typename T>
struct CoefFor;
template <>
struct CoefFor<double> {
  using type = CoefGlobal64;
};
template <>
struct CoefFor<df> {
  using type = CoefGlobalDF;
};

// One SBDF2 velocity update in one launch, transforms in T (float64, or double-float for
// the mixed path):
//   res1^ = (sigma + alpha k^2) u^ - (G u - U)^           stored as a half spectrum (float64)
//   u_out <- F^{-1}[(c1 res1^ + c0 res0^) / (sigma + alpha k^2)]   (SOLVE only)
// u_out may be u itself (the CTA reads u before it writes).  Without SOLVE (the start-up
// level) only res1^ is produced.  With ux_out set, u_x (which the matvec's packed inverse
// transform yields for free) is stored there in T, where the right-hand side of the same
// level takes it instead of transforming u again.
template <typename T, int NT, int MAXB, bool SOLVE>
__global__ void __launch_bounds__(NT, 1) k_linimp_step1d(const Inst1d* __restrict__ insts,
                                                      const int* __restrict__ ids,
                                                      cplx<double>* big,
                                                      const cplx<T>* __restrict__ tw,
                                                      const SolveRec* __restrict__ A,
                                                      const double* __restrict__ eta_all,
                                                      const double* __restrict__ hx_all,
                                                      double* __restrict__ u_all,
                                                      const double* __restrict__ U_all,
                                                      const cplx<double>* __restrict__ res0,
                                                      cplx<double>* __restrict__ res1,
                                                      double c1, double c0,
                                                      cplx<double>* __restrict__ ws,
                                                      double* __restrict__ u_out,
                                                      void* __restrict__ ux_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = big ? reinterpret_cast<cplx<T>*>(big + ((size_t)blockIdx.x << kMaxLog1d))
                     : reinterpret_cast<cplx<T>*>(smem);
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1;
  const double sigma = A[id].sigma, alpha = A[id].alpha;
  const double kunit = 2.0 * kPi / I.L;
  const long long hs = I.ws / kWsVectors;
  // u^ kept in the transforms' precision (cplx<df> and cplx<double> are both 16 bytes)
  cplx<T>* uh = reinterpret_cast<cplx<T>*>(ws + I.ws + (h + 1));
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(num<T>(u_all[I.off + j]), num<T>(0.0));
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, I.log2n, false, tw);
  for (int m = threadIdx.x; m <= h; m += NT) {
    const cplx<T> v = buf[m];
    uh[m] = mk(v.x, (m == 0 || m == h) ? num<T>(0.0) : v.y);   // real DC / Nyquist
  }
  __syncthreads();
  const Spec<T> sp = make_spec<T>(n, I.L, sigma, alpha);
  spectral_matvec<T, NT, MAXB>(
      buf, sp, I.log2n, [&](int m) { return uh[m]; },
      typename CoefFor<T>::type{eta_all + I.off, hx_all + I.off}, nullptr, tw, U_all + I.off,
      ux_out ? static_cast<T*>(ux_out) + I.off : nullptr);
  // mode m owns buf[m] and buf[n - m]: it reads both (gv_mode) before writing both
  for (int m = threadIdx.x; m <= h; m += NT) {
    const double k = (m == h) ? 0.0 : kunit * (double)m;
    const cplx<T> g = gv_mode(buf, m, n, sp.k(m));             // (G u - U)^_m
    const double sym = sigma + alpha * k * k;
    const T symT = num<T>(sym);
    cplx<double> r = mk(to_f64(uh[m].x * symT - g.x), to_f64(uh[m].y * symT - g.y));
    if (m == 0 || m == h) r.y = 0.0;
    res1[hs + m] = r;
    if (SOLVE) {
      const cplx<double> p = res0[hs + m];
      cplx<double> v = mk((c1 * r.x + c0 * p.x) / sym, (c1 * r.y + c0 * p.y) / sym);
      if (m == 0 || m == h) v.y = 0.0;
      buf[m] = mk(num<T>(v.x), num<T>(v.y));
      if (m > 0 && m < h) buf[n - m] = mk(num<T>(v.x), num<T>(-v.y));
    }
  }
  if (!SOLVE) return;
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, I.log2n, true, tw);
  const double inv_n = 1.0 / n;
  for (int j = threadIdx.x; j < n; j += NT) u_out[I.off + j] = to_f64(buf[j].x) * inv_n;
}

}  // namespace

// =======================================================================================
// Launchers
// =======================================================================================

cudaError_t twiddles_init(void* tw64, void* tw32, cudaStream_t s) {
  k_twiddles<<<kTwiddleN / 256, 256, 0, s>>>(
      static_cast<cplx<double>*>(tw64), static_cast<cplx<float>*>(tw32),
      reinterpret_cast<cplx<df>*>(static_cast<char*>(tw32) + kTw32Bytes));
  return cudaGetLastError();
}

cudaError_t launch_deriv1d(const Layout1d& lay, const void* tw64, const double* f, double* fx,
                           cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_deriv1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, f, fx);
    return cudaGetLastError();
  }, [&](int first, int num, cudaStream_t s) {
    return mr_launch_deriv(lay, first, num, f, fx, s);
  });
}

cudaError_t launch_apply_G1d(const Layout1d& lay, const void* tw64, const double* eta,
                             const double* hx, const double* u, double* Gu, cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_apply_G1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, eta, hx, u, Gu);
    return cudaGetLastError();
  }, [&](int first, int num, cudaStream_t s) {
    return mr_launch_apply_G(lay, first, num, eta, hx, u, Gu, s);
  });
}

cudaError_t launch_coeffs1d(const Layout1d& lay, const double* eta, const double* hx, int kind,
                            SolveRec* rec, cudaStream_t s) {
  k_coeffs1d<256><<<lay.count, 256, 0, s>>>(lay.d_inst, lay.d_ids, eta, hx, kind, rec);
  return cudaGetLastError();
}

cudaError_t launch_precond1d(const Layout1d& lay, const void* tw64, const SolveRec* rec,
                             const double* r, double* z, cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_precond1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, rec, r, z);
    return cudaGetLastError();
  }, [&](int first, int num, cudaStream_t s) {
    return mr_launch_precond(lay, first, num, rec, r, z, s);
  });
}

cudaError_t launch_axpy1d(const Layout1d& lay, const double* dt, double* out, const double* base,
                          int nterms, const double* const* f, const double* c, double scale,
                          cudaStream_t s) {
  AxpyArgs a{};
  a.nterms = nterms;
  for (int t = 0; t < nterms && t < 4; ++t) {
    a.f[t] = f[t];
    a.c[t] = c[t];
  }
  k_axpy1d<<<lay.count, 256, 0, s>>>(lay.d_inst, dt, out, base, a, scale);
  return cudaGetLastError();
}

cudaError_t launch_dealias1d(const Layout1d& lay, const void* tw64, const void* tw32,
                             int precision, const double* h, double* eta, double* U, double* u,
                             cudaStream_t s) {
  const bool dfp = precision == SGN_PREC_MIXED;
  const void* twT = dfp ? static_cast<const void*>(static_cast<const char*>(tw32) + kTw32Bytes)
                        : tw64;
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;    // cplx<double> and cplx<df>: 16 bytes
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto run = [&](auto kern, auto twp) -> cudaError_t {
      cudaError_t e = set_smem(kern, sm);
      if (e) return e;
      kern<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, twp, h, eta, U, u);
      return cudaGetLastError();
    };
    if (dfp) return run(k_dealias1d<df, NT, MB>, static_cast<const cplx<df>*>(twT));
    return run(k_dealias1d<double, NT, MB>, static_cast<const cplx<double>*>(twT));
  });
}

cudaError_t launch_rhs_nc1d(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, double g, const double* eta, const double* u,
                            const double* h, const double* hx, double* f_eta, double* M,
                            double* scratch, cudaStream_t s) {
  const bool dfp = precision == SGN_PREC_MIXED;
  const void* twT = dfp ? static_cast<const void*>(static_cast<const char*>(tw32) + kTw32Bytes)
                        : tw64;
  double* w1 = scratch + lay.points;
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;    // cplx<double> and cplx<df>: 16 bytes
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto run = [&](auto kern, auto twp) -> cudaError_t {
      cudaError_t e = set_smem(kern, sm);
      if (e) return e;
      kern<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, twp, g, eta, u, h, hx, f_eta,
                               M, scratch, w1);
      return cudaGetLastError();
    };
    if (dfp) return run(k_rhs_nc1d<df, NT, MB>, static_cast<const cplx<df>*>(twT));
    return run(k_rhs_nc1d<double, NT, MB>, static_cast<const cplx<double>*>(twT));
  });
}

cudaError_t launch_linimp_step1d(const Layout1d& lay, const void* tw64, const void* tw32,
                                 int precision, const SolveRec* A, const double* eta,
                                 const double* hx, double* u, const double* U,
                                 const void* res0_hat, void* res1_hat, double c1, double c0,
                                 bool solve, void* ws, double* u_out, void* ux_out,
                                 cudaStream_t s) {
  const bool dfp = precision == SGN_PREC_MIXED;
  const void* twT = dfp ? static_cast<const void*>(static_cast<const char*>(tw32) + kTw32Bytes)
                        : tw64;
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;    // cplx<double> and cplx<df>: 16 bytes
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto run = [&](auto kern, auto twp) -> cudaError_t {
      cudaError_t e = set_smem(kern, sm);
      if (e) return e;
      kern<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, twp, A, eta, hx, u, U,
                               static_cast<const cplx<double>*>(res0_hat),
                               static_cast<cplx<double>*>(res1_hat), c1, c0,
                               static_cast<cplx<double>*>(ws), u_out ? u_out : u, ux_out);
      return cudaGetLastError();
    };
    auto twd = static_cast<const cplx<double>*>(twT);
    auto twf = static_cast<const cplx<df>*>(twT);
    if (dfp)
      return solve ? run(k_linimp_step1d<df, NT, MB, true>, twf)
                   : run(k_linimp_step1d<df, NT, MB, false>, twf);
    return solve ? run(k_linimp_step1d<double, NT, MB, true>, twd)
                 : run(k_linimp_step1d<double, NT, MB, false>, twd);
  });
}

}  // namespace sgn
