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

// SBDF2: res^ = (sigma + alpha k^2) u^ - (G u - U)^  (half spectrum, float64)
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_linimp_res1d(const Inst1d* __restrict__ insts,
                                                     const int* __restrict__ ids,
                                                     cplx<double>* big,
                                                     const cplx<double>* __restrict__ tw,
                                                     const SolveRec* __restrict__ A,
                                                     const double* __restrict__ eta_all,
                                                     const double* __restrict__ hx_all,
                                                     const double* __restrict__ u_all,
                                                     const double* __restrict__ U_all,
                                                     cplx<double>* __restrict__ res,
                                                     cplx<double>* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = big ? big + ((size_t)blockIdx.x << kMaxLog1d)
                          : reinterpret_cast<cplx<double>*>(smem);
  const int id = ids[blockIdx.x];
  const Inst1d I = insts[id];
  const int n = I.n, h = n >> 1;
  const double sigma = A[id].sigma, alpha = A[id].alpha;
  const long long S = h + 1;
  cplx<double>* uh = ws + I.ws + S;
  cplx<double>* out = res + I.ws / kWsVectors;
  // u^ from a transform of u alone; U enters inside the matvec (w - U, so the matvec yields
  // (G u - U)^).  Packed as u + i U, u^ would carry U's rounding (~eps ||U||), and U = G u
  // can outweigh u by eta^3 k^2 / 3, which the right-hand side's third derivatives pass on.
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = mk(u_all[I.off + j], 0.0);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, I.log2n, false, tw);
  for (int m = threadIdx.x; m <= h; m += NT)
    uh[m] = (m == 0 || m == h) ? mk(buf[m].x, 0.0) : buf[m];   // real modes of a real field
  __syncthreads();
  const Spec<double> sp = make_spec<double>(n, I.L, sigma, alpha);
  spectral_matvec<double, NT, MAXB>(buf, sp, I.log2n, [&](int m) { return uh[m]; },
                                    CoefGlobal64{eta_all + I.off, hx_all + I.off}, nullptr, tw,
                                    U_all + I.off);
  for (int m = threadIdx.x; m <= h; m += NT) {
    double k = sp.k(m);
    cplx<double> gu = gv_mode(buf, m, n, k);       // (G u - U)^_m
    out[m] = uh[m] * (sigma + alpha * k * k) - gu;
  }
}

// SBDF2: u = F^{-1}[(c1 res1^ + c0 res0^) / (sigma + alpha k^2)]
template <int NT, int MAXB>
__global__ void __launch_bounds__(NT, 1) k_linimp_solve1d(const Inst1d* __restrict__ insts,
                                                       const int* __restrict__ ids,
                                                       cplx<double>* big,
                                                       const cplx<double>* __restrict__ tw,
                                                       const SolveRec* __restrict__ A,
                                                       const cplx<double>* __restrict__ res1,
                                                       const cplx<double>* __restrict__ res0,
                                                       double c1, double c0,
                                                       double* __restrict__ u_all) {
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<double>* buf = big ? big + ((size_t)blockIdx.x << kMaxLog1d)
                          : reinterpret_cast<cplx<double>*>(smem);
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
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_deriv1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, f, fx);
    return cudaGetLastError();
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
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_linimp_res1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, A, eta, hx, u, U,
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
    const bool gl = l > kSmemLog1d;                // transform buffer in global scratch
    const size_t sm = gl ? 0 : (size_t)16 << l;
    cplx<double>* big = gl ? static_cast<cplx<double>*>(lay.big) : nullptr;
    auto k = k_linimp_solve1d<NT, MB>;
    cudaError_t e = set_smem(k, sm);
    if (e) return e;
    k<<<num, NT, sm, s>>>(lay.d_inst, lay.d_ids + first, big, tw, A,
                          static_cast<const cplx<double>*>(res1_hat),
                          static_cast<const cplx<double>*>(res0_hat), c1, c0, u);
    return cudaGetLastError();
  });
}

}  // namespace sgn
