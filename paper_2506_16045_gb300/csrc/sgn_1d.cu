// 1d periodic SGN kernels: one CTA owns one instance (n <= 8192) and keeps the whole
// transform in shared memory, so a PCG solve never leaves the SM between iterations.
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
                                                const cplx<double>* __restrict__ tw,
                                                const double* __restrict__ f,
                                                double* __restrict__ fx) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem);
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
                                                  const cplx<double>* __restrict__ tw,
                                                  const double* __restrict__ eta,
                                                  const double* __restrict__ hx,
                                                  const double* __restrict__ u,
                                                  double* __restrict__ Gu) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n, h = n >> 1;
  const double kunit = 2.0 * kPi / I.L;
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
                                                  const cplx<double>* __restrict__ tw,
                                                  const SolveRec* __restrict__ rec,
                                                  const double* __restrict__ r,
                                                  double* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem);
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

// a7: right-hand side of Eq:DAE_DSWE with F from Def:bigF, in number type T (float64 for
// the float64 path, double-float for the mixed path): four derivative pairs
// (u, eta u) -> (d, m); (zeta, s) -> (zeta_x, s_x); d -> d_x; Phi' -> Phi'_x with
// Phi' = eta^3 Q/3 + eta^2 m d + eta^2 S/2 + eta m s - eta u^2 (the flux -(eta u^2)_x folded
// in), Q = u d_x - d^2, S = u s_x (reading R6), and
// f_eta = -m, f_U = -g eta zeta_x + Phi'_x - h_x Psi, Psi = eta^2 Q/2 + eta m d + eta S + m s.
template <typename T, int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_rhs1d(const Inst1d* __restrict__ insts,
                                              const int* __restrict__ ids,
                                              const cplx<T>* __restrict__ tw, double g,
                                              const double* __restrict__ eta_all,
                                              const double* __restrict__ u_all,
                                              const double* __restrict__ h_all,
                                              const double* __restrict__ hx_all,
                                              double* __restrict__ fe_all,
                                              double* __restrict__ fU_all,
                                              double* __restrict__ scratch, long long P) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem);
  const Inst1d I = insts[ids[blockIdx.x]];
  const int n = I.n, log2n = I.log2n;
  const T kn = num<T>(2.0 * kPi / I.L / (double)n);
  const T third = num<T>(1.0 / 3.0);
  const T gT = num<T>(g);
  const double* eta = eta_all + I.off;
  const double* u = u_all + I.off;
  const double* hh = h_all + I.off;
  const double* hx = hx_all + I.off;
  // scratch planes hold T values (8 bytes each for double and double-float)
  T* sd = reinterpret_cast<T*>(scratch + I.off);           // d = u_x
  T* sm = reinterpret_cast<T*>(scratch + P + I.off);       // m = (eta u)_x
  T* szx = reinterpret_cast<T*>(scratch + 2 * P + I.off);  // zeta_x
  T* ssx = reinterpret_cast<T*>(scratch + 3 * P + I.off);  // s_x, s = h_x u
  T* spsi = reinterpret_cast<T*>(scratch + 4 * P + I.off); // Psi
  deriv_pair<T, NT, MAXB>(buf, n, log2n, kn, [&](int j) {
    T uj = num<T>(u[j]);
    return mk(uj, num<T>(eta[j]) * uj);
  }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    sd[j] = buf[j].x;
    sm[j] = buf[j].y;
  }
  __syncthreads();
  deriv_pair<T, NT, MAXB>(buf, n, log2n, kn, [&](int j) {
    return mk(num<T>(eta[j] - hh[j]), num<T>(hx[j]) * num<T>(u[j]));
  }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    szx[j] = buf[j].x;
    ssx[j] = buf[j].y;
  }
  __syncthreads();
  deriv_pair<T, NT, MAXB>(buf, n, log2n, kn, [&](int j) { return mk(sd[j], from_int<T>(0)); },
                          tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    T e = num<T>(eta[j]), uj = num<T>(u[j]), d = sd[j], m = sm[j];
    T s = num<T>(hx[j]) * uj;
    T Q = uj * buf[j].x - d * d;
    T Sv = uj * ssx[j];
    T e2 = e * e;
    T md = m * d;
    T Phi = e2 * e * Q * third + e2 * md + half(e2 * Sv) + e * m * s - e * uj * uj;
    spsi[j] = half(e2 * Q) + e * md + e * Sv + m * s;
    buf[j] = mk(Phi, from_int<T>(0));
  }
  __syncthreads();
  deriv_pair<T, NT, MAXB>(buf, n, log2n, kn, [&](int j) { return buf[j]; }, tw);
  for (int j = threadIdx.x; j < n; j += NT) {
    fe_all[I.off + j] = -to_f64(sm[j]);
    T fU = buf[j].x - gT * num<T>(eta[j]) * szx[j] - num<T>(hx[j]) * spsi[j];
    fU_all[I.off + j] = to_f64(fU);
  }
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

// SBDF2: res^ = (sigma + alpha k^2) u^ - (G u)^ + U^  (half spectrum, float64)
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_linimp_res1d(const Inst1d* __restrict__ insts,
                                                     const int* __restrict__ ids,
                                                     const cplx<double>* __restrict__ tw,
                                                     const SolveRec* __restrict__ A,
                                                     const double* __restrict__ eta_all,
                                                     const double* __restrict__ hx_all,
                                                     const double* __restrict__ u_all,
                                                     const double* __restrict__ U_all,
                                                     cplx<double>* __restrict__ res,
                                                     cplx<double>* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem);
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1;
  const double kunit = 2.0 * kPi / I.L;
  const double sigma = A[id].sigma, alpha = A[id].alpha;
  const long long S = h + 1;
  cplx<double>* Uh = ws + I.ws;
  cplx<double>* uh = ws + I.ws + S;
  cplx<double>* out = res + I.ws / kWsVectors;
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(u_all[I.off + j], U_all[I.off + j]);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, false, tw);
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<double> z = buf[m], zc = conj(buf[(n - m) & (n - 1)]);
    uh[m] = (z + zc) * 0.5;
    Uh[m] = mul_mi(z - zc) * 0.5;
  }
  __syncthreads();
  const Spec<double> sp = make_spec<double>(n, I.L, sigma, alpha);
  spectral_matvec<double, NT, MAXB>(buf, sp, I.log2n, [&](int m) { return uh[m]; },
                                    CoefGlobal64{eta_all + I.off, hx_all + I.off}, nullptr, tw);
  for (int m = threadIdx.x; m <= h; m += NT) {
    double k = sp.k(m);
    cplx<double> gu = gv_mode(buf, m, n, k);
    out[m] = uh[m] * (sigma + alpha * k * k) - gu + Uh[m];
  }
}

// SBDF2: u = F^{-1}[(c1 res1^ + c0 res0^) / (sigma + alpha k^2)]
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_linimp_solve1d(const Inst1d* __restrict__ insts,
                                                       const int* __restrict__ ids,
                                                       const cplx<double>* __restrict__ tw,
                                                       const SolveRec* __restrict__ A,
                                                       const cplx<double>* __restrict__ res1,
                                                       const cplx<double>* __restrict__ res0,
                                                       double c1, double c0,
                                                       double* __restrict__ u_all) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem);
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1;
  const double kunit = 2.0 * kPi / I.L;
  const double sigma = A[id].sigma, alpha = A[id].alpha;
  const long long hs = I.ws / kWsVectors;
  for (int m = threadIdx.x; m <= h; m += NT) {
    double k = (m == h) ? 0.0 : kunit * (double)m;
    cplx<double> v = (res1[hs + m] * c1 + res0[hs + m] * c0) * (1.0 / (sigma + alpha * k * k));
    buf[m] = v;
    if (m > 0 && m < h) buf[n - m] = conj(v);
  }
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, true, tw);
  const double inv_n = 1.0 / n;
  for (int j = threadIdx.x; j < n; j += NT) u_all[I.off + j] = buf[j].x * inv_n;
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
    size_t sm = (size_t)16 << l;
    auto k = k_deriv1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tw, f, fx);
    return cudaGetLastError();
  });
}

cudaError_t launch_apply_G1d(const Layout1d& lay, const void* tw64, const double* eta,
                             const double* hx, const double* u, double* Gu, cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    size_t sm = (size_t)16 << l;
    auto k = k_apply_G1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tw, eta, hx, u, Gu);
    return cudaGetLastError();
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
    size_t sm = (size_t)16 << l;
    auto k = k_precond1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tw, rec, r, z);
    return cudaGetLastError();
  });
}

cudaError_t launch_rhs1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         double g, const double* eta, const double* u, const double* h,
                         const double* hx, double* f_eta, double* f_U, double* scratch,
                         cudaStream_t s) {
  auto t64 = static_cast<const cplx<double>*>(tw64);
  auto tdf = reinterpret_cast<const cplx<df>*>(static_cast<const char*>(tw32) + kTw32Bytes);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    size_t sm = (size_t)16 << l;
    if (precision == SGN_PREC_MIXED) {
      auto k = k_rhs1d<df, NT, MB>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tdf, g, eta, u, h, hx, f_eta, f_U,
                            scratch, lay.points);
    } else {
      auto k = k_rhs1d<double, NT, MB>;
      cudaError_t e = set_smem(k, sm);
      if (e) return e;
      k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, t64, g, eta, u, h, hx, f_eta, f_U,
                            scratch, lay.points);
    }
    return cudaGetLastError();
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

cudaError_t launch_linimp_res1d(const Layout1d& lay, const void* tw64, const SolveRec* A,
                                   const double* eta, const double* hx, const double* u,
                                   const double* U, void* res_hat, void* ws, cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    size_t sm = (size_t)16 << l;
    auto k = k_linimp_res1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tw, A, eta, hx, u, U,
                          static_cast<cplx<double>*>(res_hat), static_cast<cplx<double>*>(ws));
    return cudaGetLastError();
  });
}

cudaError_t launch_linimp_solve1d(const Layout1d& lay, const void* tw64, const SolveRec* A,
                                  const void* res1_hat, const void* res0_hat, double c1,
                                  double c0, double* u, cudaStream_t s) {
  auto tw = static_cast<const cplx<double>*>(tw64);
  return for_each_class(lay, s, [&](auto NTc, auto MBc, int l, int first, int num, cudaStream_t s) {
    constexpr int NT = decltype(NTc)::value, MB = decltype(MBc)::value;
    size_t sm = (size_t)16 << l;
    auto k = k_linimp_solve1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, tw, A,
                          static_cast<const cplx<double>*>(res1_hat),
                          static_cast<const cplx<double>*>(res0_hat), c1, c0, u);
    return cudaGetLastError();
  });
}

}  // namespace sgn
