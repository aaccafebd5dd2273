// 1d instances whose n is not a power of two: n = 2^a 3^b 5^c (a >= 1, 6 <= n <= 6144), the
// grids of §6.1 at sizes the register-blocked power-of-two kernels do not take.  One CTA of
// kMrNT threads per instance, with a mixed-radix Stockham FFT in shared memory (radices 8,
// 4, 2 for the power of two, then 5 and 3), two buffers used in turn, and per-size twiddle
// tables built when the layout is created.  Every spectral operation follows the same
// formulas as the power-of-two kernels (D = F^{-1}(iK)F with the n/2 wavenumber set to 0,
// Def:G in its weak form, A^{-1} per mode, PCG with the stopping rule R7, the right-hand
// side of Eq:DAE_DSWE with Def:bigF):
//   k_mr_deriv   f -> D f                                   (float64)
//   k_mr_apply_G u -> G u                                   (float64)
//   k_mr_precond r -> A^{-1} r                              (float64)
//   k_mr_pcg     G x = b: float64 PCG, or float32 inner PCG inside double-float refinement
//   k_mr_rhs     (f_eta, f_U)                               (float64 or double-float)
#include <vector>

#include "sgn_1d_dev.cuh"
#include "sgn_mr_fft.cuh"

namespace sgn {
namespace {

using d1::kPi;
using mr::MrPlan;
using mr::mr_plan;
using mr::k_mr_twiddles;
constexpr int kMrNT = 256;
constexpr int kMrMaxN = 16384;       // largest generic n
constexpr int kMrSmemN = 6144;       // largest n whose two transform buffers (192 KB) are in
                                     // shared memory; above it they are in global memory

// wavenumber of mode m (Nyquist 0), in T
template <typename T>
__device__ __forceinline__ T mr_k(int m, int n, double kunit) {
  return num<T>(kunit * (double)wave_index(m, n));
}

struct MrTw {            // the instance's twiddle tables (n - 1 entries each)
  const cplx<double>* d;
  const cplx<float>* f;
  const cplx<df>* h;
};
template <typename T>
__device__ __forceinline__ const cplx<T>* tw_of(const MrTw& t);
template <>
__device__ __forceinline__ const cplx<double>* tw_of<double>(const MrTw& t) { return t.d; }
template <>
__device__ __forceinline__ const cplx<float>* tw_of<float>(const MrTw& t) { return t.f; }
template <>
__device__ __forceinline__ const cplx<df>* tw_of<df>(const MrTw& t) { return t.h; }

struct MrArgs {
  const Inst1d* insts;
  const int* ids;          // the generic instances' ids
  cplx<double>* big;       // global transform buffers of the instances above kMrSmemN
  const cplx<double>* tw64;
  const cplx<float>* tw32;
  const cplx<df>* twdf;
};

__device__ __forceinline__ MrTw mr_tw(const MrArgs& A, const Inst1d& I) {
  return MrTw{A.tw64 + I.tw, A.tw32 + I.tw, A.twdf + I.tw};
}

// The instance's two transform buffers (n entries of 16 bytes each): shared memory, or its
// slot of the layout's global buffer (I.gbuf >= 0, n > kMrSmemN; the CTA's own L2-resident
// copy, written and read by this CTA only, ordered by the same barriers).
template <typename T>
__device__ __forceinline__ cplx<T>* tbuf(const MrArgs& A, const Inst1d& I, int which) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* base = I.gbuf >= 0 ? reinterpret_cast<unsigned char*>(A.big + I.gbuf) : smem;
  return reinterpret_cast<cplx<T>*>(base + (size_t)which * 16 * I.n);
}

// f_x of the real fields a + i b packed in buf (transform, i k / n, inverse): re / im
template <typename T>
__device__ __forceinline__ cplx<T>* mr_deriv_pair(cplx<T>* A, cplx<T>* B, const MrPlan& P,
                                                  double kunit, const cplx<T>* tw) {
  const int n = P.n;
  cplx<T>* F = mr::mr_fft<T, kMrNT>(A, B, P, false, tw);
  const double inv_n = 1.0 / n;
  for (int m = threadIdx.x; m < n; m += kMrNT) F[m] = mul_pi(F[m]) * num<T>(kunit * wave_index(m, n) * inv_n);
  __syncthreads();
  return mr::mr_fft<T, kMrNT>(F, F == A ? B : A, P, true, tw);
}

// ---- operators (float64) ----------------------------------------------------------------
__global__ void __launch_bounds__(kMrNT) k_mr_deriv(const MrArgs A, const double* __restrict__ f,
                                                   double* __restrict__ fx) {
  const Inst1d I = A.insts[A.ids[blockIdx.x]];
  MrPlan P;
  mr_plan(I.n, P);
  cplx<double>* a = tbuf<double>(A, I, 0);
  cplx<double>* b = tbuf<double>(A, I, 1);
  for (int j = threadIdx.x; j < I.n; j += kMrNT) a[j] = mk(f[I.off + j], 0.0);
  __syncthreads();
  const cplx<double>* o = mr_deriv_pair<double>(a, b, P, 2.0 * kPi / I.L, mr_tw(A, I).d);
  for (int j = threadIdx.x; j < I.n; j += kMrNT) fx[I.off + j] = o[j].x;
}

// (G v)^ of a real field held as its full spectrum V (modes 0..n-1): the transform of
// v + i v_x is (1 - k) V; pointwise w = c1 v + c2 v_x, q = c2 v + c3 v_x; (G v)^_m =
// ((1 - k_m) Y_m + (1 + k_m) conj Y_{n-m}) / 2 with Y the transform of w + i q (Def:G as
// w - q_x).  Writes the half spectrum m = 0..n/2 of G v into out (T arithmetic).  c: the
// coefficients c1, c2, c3 at point j.
template <typename T, typename Coef>
__device__ void mr_matvec(cplx<T>* a, cplx<T>* b, const MrPlan& P, double kunit,
                          const cplx<T>* tw, Coef coef, cplx<T>* out) {
  const int n = P.n, h = n / 2;
  // a holds V (full spectrum); form (1 - k) V in place
  for (int m = threadIdx.x; m < n; m += kMrNT) a[m] = a[m] * (num<T>(1.0) - mr_k<T>(m, n, kunit));
  __syncthreads();
  cplx<T>* z = mr::mr_fft<T, kMrNT>(a, b, P, true, tw);
  const T inv_n = num<T>(1.0 / n);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T v = z[j].x * inv_n, vx = z[j].y * inv_n;
    T c1, c2, c3;
    coef(j, c1, c2, c3);
    z[j] = mk(c1 * v + c2 * vx, c2 * v + c3 * vx);
  }
  __syncthreads();
  cplx<T>* Y = mr::mr_fft<T, kMrNT>(z, z == a ? b : a, P, false, tw);
  for (int m = threadIdx.x; m <= h; m += kMrNT) {
    const T k = mr_k<T>(m, n, kunit);
    const cplx<T> y = Y[m], ym = conj(Y[(n - m) % n]);
    const cplx<T> s = y * (num<T>(1.0) - k) + ym * (num<T>(1.0) + k);
    out[m] = mk(half(s.x), half(s.y));
  }
  __syncthreads();
}

struct Coef64 {
  const double* eta;
  const double* hx;
  __device__ void operator()(int j, double& c1, double& c2, double& c3) const {
    const double e = eta[j], g = hx[j];
    c1 = e * (1.0 + g * g);
    c2 = 0.5 * e * e * g;
    c3 = e * e * e / 3.0;
  }
};

__global__ void __launch_bounds__(kMrNT) k_mr_apply_G(const MrArgs A, const double* __restrict__ eta,
                                                     const double* __restrict__ hx,
                                                     const double* __restrict__ u,
                                                     double* __restrict__ Gu) {
  const Inst1d I = A.insts[A.ids[blockIdx.x]];
  MrPlan P;
  mr_plan(I.n, P);
  const int n = I.n, h = n / 2;
  cplx<double>* a = tbuf<double>(A, I, 0);
  cplx<double>* b = tbuf<double>(A, I, 1);
  const cplx<double>* tw = mr_tw(A, I).d;
  const double kunit = 2.0 * kPi / I.L;
  for (int j = threadIdx.x; j < n; j += kMrNT) a[j] = mk(u[I.off + j], 0.0);
  __syncthreads();
  cplx<double>* V = mr::mr_fft<double, kMrNT>(a, b, P, false, tw);
  cplx<double>* o = V == a ? b : a;
  // (G u)^ of modes 0..n/2 into V itself: mode m is read and written only by the thread
  // that computes it (its mirror n - m is above n/2 and never written)
  mr_matvec<double>(V, o, P, kunit, tw, Coef64{eta + I.off, hx + I.off}, V);
  // V[0..h] = (G u)^; build the Hermitian full spectrum and invert
  for (int m = threadIdx.x; m < h; m += kMrNT)
    if (m > 0) V[n - m] = conj(V[m]);
  __syncthreads();
  const cplx<double>* x = mr::mr_fft<double, kMrNT>(V, o, P, true, tw);
  for (int j = threadIdx.x; j < n; j += kMrNT) Gu[I.off + j] = x[j].x / n;
}

__global__ void __launch_bounds__(kMrNT) k_mr_precond(const MrArgs A, const SolveRec* __restrict__ rec,
                                                     const double* __restrict__ r,
                                                     double* __restrict__ z) {
  const int id = A.ids[blockIdx.x];
  const Inst1d I = A.insts[id];
  MrPlan P;
  mr_plan(I.n, P);
  const int n = I.n;
  cplx<double>* a = tbuf<double>(A, I, 0);
  cplx<double>* b = tbuf<double>(A, I, 1);
  const cplx<double>* tw = mr_tw(A, I).d;
  const double kunit = 2.0 * kPi / I.L, sigma = rec[id].sigma, alpha = rec[id].alpha;
  for (int j = threadIdx.x; j < n; j += kMrNT) a[j] = mk(r[I.off + j], 0.0);
  __syncthreads();
  cplx<double>* F = mr::mr_fft<double, kMrNT>(a, b, P, false, tw);
  for (int m = threadIdx.x; m < n; m += kMrNT) {
    const double k = kunit * wave_index(m, n);
    F[m] = F[m] * (1.0 / ((sigma + alpha * k * k) * (double)n));
  }
  __syncthreads();
  const cplx<double>* x = mr::mr_fft<double, kMrNT>(F, F == a ? b : a, P, true, tw);
  for (int j = threadIdx.x; j < n; j += kMrNT) z[I.off + j] = x[j].x;
}

// ---- PCG -------------------------------------------------------------------------------
struct MrPcgArgs {
  const double* eta;
  const double* hx;
  const double* b;
  double* x;
  const SolveRec* given;
  int kind;
  double rtol, rtol_inner;
  int maxit, max_refine;
  SolveRec* rec;
  cplx<double>* ws;
};

// coefficients of Def:MatrixM in double-float and float32
struct CoefDf {
  const double* eta;
  const double* hx;
  __device__ void operator()(int j, df& c1, df& c2, df& c3) const {
    const df e(eta[j]), g(hx[j]);
    const df e2 = e * e;
    c1 = e + e * g * g;
    c2 = half(e2 * g);
    c3 = e2 * e * df(1.0 / 3.0);
  }
};
struct Coef32 {
  const double* eta;
  const double* hx;
  __device__ void operator()(int j, float& c1, float& c2, float& c3) const {
    const float e = (float)eta[j], g = (float)hx[j];
    c1 = e * (1.0f + g * g);
    c2 = 0.5f * e * e * g;
    c3 = e * e * e * (1.0f / 3.0f);
  }
};

// the full spectrum V_m (m = 0..n-1) of a real field from its half spectrum H (m = 0..n/2),
// the DC and Nyquist coefficients taken real (their imaginary parts are rounding residue)
template <typename T>
__device__ __forceinline__ void mr_full(cplx<T>* V, const cplx<T>* H, int n) {
  const int h = n / 2;
  for (int m = threadIdx.x; m < n; m += kMrNT) {
    cplx<T> v;
    if (m == 0 || m == h) v = mk(H[m].x, from_int<T>(0));
    else if (m < h) v = H[m];
    else v = conj(H[n - m]);
    V[m] = v;
  }
  __syncthreads();
}

template <bool MIXED>
__global__ void __launch_bounds__(kMrNT) k_mr_pcg(const MrArgs A, const MrPcgArgs a) {
  __shared__ double red[kMrNT / 32 + 1];
  const int id = A.ids[blockIdx.x];
  const Inst1d I = A.insts[id];
  MrPlan P;
  mr_plan(I.n, P);
  const int n = I.n, h = n / 2;
  const long long S = h + 1;
  const double kunit = 2.0 * kPi / I.L;
  const MrTw tws = mr_tw(A, I);
  const double* eta = a.eta + I.off;
  const double* hx = a.hx + I.off;
  // ---- a1: coefficients (or the caller's)
  SolveRec R = {};
  if (a.given) {
    R = a.given[id];
    R.status = SGN_OK;
  } else {
    d1::coeffs_block<kMrNT>(eta, hx, n, a.kind, red, R);
  }
  R.iters = 0;
  R.refinements = 0;
  R.ratio = 0.0;
  if (R.status != SGN_OK) {
    if (threadIdx.x == 0) a.rec[id] = R;
    return;
  }
  const double sigma = R.sigma, alpha = R.alpha;
  auto dinv = [&](int m) {
    const double k = kunit * wave_index(m, n);
    return 1.0 / (sigma + alpha * k * k);
  };
  auto wgt = [&](int m) { return (m == 0 || m == h) ? 1.0 : 2.0; };
  cplx<double>* ws = a.ws + I.ws;
  // ---- b^ and x0^ from one transform of b + i x0 (float64)
  cplx<double>* d0 = tbuf<double>(A, I, 0);
  cplx<double>* d1 = tbuf<double>(A, I, 1);
  for (int j = threadIdx.x; j < n; j += kMrNT) d0[j] = mk(a.b[I.off + j], a.x[I.off + j]);
  __syncthreads();
  cplx<double>* Y = mr::mr_fft<double, kMrNT>(d0, d1, P, false, tws.d);
  cplx<double>* Bh = ws;            // float64 path: b^, x^, r^, p^, (G p)^ in slots 0..4
  cplx<double>* Xh = ws + S;
  double bb = 0.0;
  for (int m = threadIdx.x; m <= h; m += kMrNT) {
    const cplx<double> y = Y[m], ym = conj(Y[(n - m) % n]);
    const cplx<double> sb = y + ym, sx = mul_mi(y - ym);
    const cplx<double> bh = mk(0.5 * sb.x, 0.5 * sb.y), xh = mk(0.5 * sx.x, 0.5 * sx.y);
    Bh[m] = bh;
    Xh[m] = xh;
    bb += wgt(m) * (bh.x * bh.x + bh.y * bh.y) * dinv(m);
  }
  bb = block_sum<kMrNT>(bb, red);
  const double bnorm = sqrt(bb);
  if (!(bnorm > 0.0)) {
    for (int j = threadIdx.x; j < n; j += kMrNT) a.x[I.off + j] = 0.0;
    R.status = (bb == 0.0) ? SGN_OK : SGN_ERR_BREAKDOWN;
    if (threadIdx.x == 0) a.rec[id] = R;
    return;
  }
  int iters = 0, status = SGN_OK;
  if constexpr (!MIXED) {
    cplx<double>* Rh = ws + 2 * S;
    cplx<double>* Ph = ws + 3 * S;
    cplx<double>* Gh = ws + 4 * S;
    const Coef64 coef{eta, hx};
    auto matvec = [&](const cplx<double>* Vh) {     // Gh = (G v)^
      mr_full<double>(d0, Vh, n);
      mr_matvec<double>(d0, d1, P, kunit, tws.d, coef, Gh);
    };
    matvec(Xh);
    double rz = 0.0;
    for (int m = threadIdx.x; m <= h; m += kMrNT) {
      const cplx<double> r = Bh[m] - Gh[m];
      Rh[m] = r;
      Ph[m] = r * dinv(m);
      rz += wgt(m) * (r.x * r.x + r.y * r.y) * dinv(m);
    }
    rz = block_sum<kMrNT>(rz, red);
    const double tol = a.rtol * bnorm;
    while (sqrt(rz) > tol) {
      if (iters >= a.maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      __syncthreads();
      matvec(Ph);
      double pq = 0.0;
      for (int m = threadIdx.x; m <= h; m += kMrNT)
        pq += wgt(m) * (Ph[m].x * Gh[m].x + Ph[m].y * Gh[m].y);
      pq = block_sum<kMrNT>(pq, red);
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double al = rz / pq;
      double rzn = 0.0;
      for (int m = threadIdx.x; m <= h; m += kMrNT) {
        Xh[m] = Xh[m] + Ph[m] * al;
        const cplx<double> r = Rh[m] - Gh[m] * al;
        Rh[m] = r;
        rzn += wgt(m) * (r.x * r.x + r.y * r.y) * dinv(m);
      }
      rzn = block_sum<kMrNT>(rzn, red);
      ++iters;
      if (!isfinite(rzn)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double be = rzn / rz;
      rz = rzn;
      for (int m = threadIdx.x; m <= h; m += kMrNT) Ph[m] = Rh[m] * dinv(m) + Ph[m] * be;
    }
    R.ratio = sqrt(rz) / bnorm;
    __syncthreads();
    mr_full<double>(d0, Xh, n);
    const cplx<double>* x = mr::mr_fft<double, kMrNT>(d0, d1, P, true, tws.d);
    for (int j = threadIdx.x; j < n; j += kMrNT) a.x[I.off + j] = x[j].x / n;
  } else {
    // double-float refinement: b^ and x^ (slots 0, 1) and the residual (slot 4) in
    // double-float; the float32 inner solve's r, p (slot 2) and d, G p (slot 3), two
    // float32 vectors per slot
    cplx<df>* Bd = reinterpret_cast<cplx<df>*>(ws);
    cplx<df>* Xd = reinterpret_cast<cplx<df>*>(ws + S);
    cplx<df>* Gd = reinterpret_cast<cplx<df>*>(ws + 4 * S);
    cplx<float>* Rf = reinterpret_cast<cplx<float>*>(ws + 2 * S);
    cplx<float>* Pf = Rf + S;
    cplx<float>* Df = reinterpret_cast<cplx<float>*>(ws + 3 * S);
    cplx<float>* Gf = Df + S;
    // the float64 b^, x^ become double-float (each thread rewrites its own modes in place)
    for (int m = threadIdx.x; m <= h; m += kMrNT) {
      const cplx<double> bh = Bh[m], xh = Xh[m];
      Bd[m] = mk(df(bh.x), df(bh.y));
      Xd[m] = mk(df(xh.x), df(xh.y));
    }
    __syncthreads();
    cplx<df>* h0 = tbuf<df>(A, I, 0);
    cplx<df>* h1 = tbuf<df>(A, I, 1);
    cplx<float>* f0 = tbuf<float>(A, I, 0);
    cplx<float>* f1 = tbuf<float>(A, I, 1);
    const CoefDf cdf{eta, hx};
    const Coef32 c32{eta, hx};
    const float sigf = (float)sigma, alf = (float)alpha, kf = (float)kunit;
    auto dinvf = [&](int m) {
      const float k = kf * (float)wave_index(m, n);
      return 1.0f / (sigf + alf * k * k);
    };
    int refinements = 0;
    double ratio = 0.0;
    for (;;) {
      // r^ = b^ - (G x)^ in double-float, and r.A^{-1}r
      mr_full<df>(h0, Xd, n);
      mr_matvec<df>(h0, h1, P, kunit, tws.h, cdf, Gd);
      double rz64 = 0.0;
      for (int m = threadIdx.x; m <= h; m += kMrNT) {
        const cplx<df> r = Bd[m] - Gd[m];
        Gd[m] = r;
        const double rx = to_f64(r.x), ry = to_f64(r.y);
        rz64 += wgt(m) * (rx * rx + ry * ry) * dinv(m);
      }
      rz64 = block_sum<kMrNT>(rz64, red);
      const double nr = sqrt(rz64);
      ratio = nr / bnorm;
      if (ratio <= a.rtol) {
        status = SGN_OK;
        break;
      }
      if (status != SGN_OK) break;
      if (refinements >= a.max_refine || iters >= a.maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      const double tin = a.rtol_inner > 0.0 ? a.rtol_inner
                                            : fmin(0.1, fmax(1e-6, 0.3 * a.rtol / ratio));
      const float sc = (float)(1.0 / nr);
      // float32 PCG for G d = r / ||r||
      double rz = 0.0;
      for (int m = threadIdx.x; m <= h; m += kMrNT) {
        const cplx<float> r = mk((float)to_f64(Gd[m].x) * sc, (float)to_f64(Gd[m].y) * sc);
        Rf[m] = r;
        Df[m] = mk(0.0f, 0.0f);
        const cplx<float> z = r * dinvf(m);
        Pf[m] = z;
        rz += wgt(m) * (double)(r.x * z.x + r.y * z.y);
      }
      rz = block_sum<kMrNT>(rz, red);
      const int it0 = iters;
      int st_in = SGN_OK;
      while (sqrt(rz) > tin) {
        if (iters >= a.maxit) {
          st_in = SGN_ERR_NOT_CONVERGED;
          break;
        }
        __syncthreads();
        mr_full<float>(f0, Pf, n);
        mr_matvec<float>(f0, f1, P, kunit, tws.f, c32, Gf);
        double pq = 0.0;
        for (int m = threadIdx.x; m <= h; m += kMrNT)
          pq += wgt(m) * (double)(Pf[m].x * Gf[m].x + Pf[m].y * Gf[m].y);
        pq = block_sum<kMrNT>(pq, red);
        if (!(pq > 0.0) || !isfinite(pq)) {
          st_in = SGN_ERR_BREAKDOWN;
          break;
        }
        const float al = (float)(rz / pq);
        double rzn = 0.0;
        for (int m = threadIdx.x; m <= h; m += kMrNT) {
          Df[m] = Df[m] + Pf[m] * al;
          const cplx<float> r = Rf[m] - Gf[m] * al;
          Rf[m] = r;
          rzn += wgt(m) * (double)((r.x * r.x + r.y * r.y) * dinvf(m));
        }
        rzn = block_sum<kMrNT>(rzn, red);
        ++iters;
        if (!isfinite(rzn)) {
          st_in = SGN_ERR_BREAKDOWN;
          break;
        }
        const float be = (float)(rzn / rz);
        rz = rzn;
        for (int m = threadIdx.x; m <= h; m += kMrNT) Pf[m] = Rf[m] * dinvf(m) + Pf[m] * be;
      }
      // a float32 breakdown after some progress keeps the correction (the next residual
      // decides); the iteration cap is reported by the refinement loop
      if (st_in == SGN_ERR_BREAKDOWN && iters == it0) status = SGN_ERR_BREAKDOWN;
      const df un(nr);
      __syncthreads();
      for (int m = threadIdx.x; m <= h; m += kMrNT)
        Xd[m] = mk(Xd[m].x + df(Df[m].x, 0.0f) * un, Xd[m].y + df(Df[m].y, 0.0f) * un);
      ++refinements;
      __syncthreads();
    }
    R.refinements = refinements;
    R.ratio = ratio;
    __syncthreads();
    mr_full<df>(h0, Xd, n);
    const cplx<df>* x = mr::mr_fft<df, kMrNT>(h0, h1, P, true, tws.h);
    const df inv_n(1.0 / n);
    for (int j = threadIdx.x; j < n; j += kMrNT) a.x[I.off + j] = to_f64(x[j].x * inv_n);
  }
  R.iters = iters;
  R.status = status;
  if (threadIdx.x == 0) a.rec[id] = R;
}

// ---- right-hand side (Eq:DAE_DSWE with Def:bigF, reading R6) ----------------------------
// Derivative pairs (u, eta u) -> (d, m); (zeta, s) -> (zeta_x, s_x); d -> d_x; Phi' -> Phi'_x
// with Phi' = eta^3 Q/3 + eta^2 m d + eta^2 S/2 + eta m s - eta u^2 (the flux folded in),
// Q = u d_x - d^2, S = u s_x; f_eta = -m, f_U = -g eta zeta_x + Phi'_x - h_x Psi,
// Psi = eta^2 Q/2 + eta m d + eta S + m s.  Intermediates in scratch planes (T per point).
template <typename T>
__global__ void __launch_bounds__(kMrNT) k_mr_rhs(const MrArgs A, double g, const double* __restrict__ eta,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ hgt,
                                                 const double* __restrict__ hx,
                                                 double* __restrict__ f_eta, double* __restrict__ f_U,
                                                 double* __restrict__ scr, long long Ptot) {
  const Inst1d I = A.insts[A.ids[blockIdx.x]];
  MrPlan P;
  mr_plan(I.n, P);
  const int n = I.n;
  const long long o = I.off;
  const double kunit = 2.0 * kPi / I.L;
  const cplx<T>* tw = tw_of<T>(mr_tw(A, I));
  cplx<T>* b0 = tbuf<T>(A, I, 0);
  cplx<T>* b1 = tbuf<T>(A, I, 1);
  // planes of Ptot 8-byte values (float64 or double-float), indexed by point
  T* D = reinterpret_cast<T*>(scr);                 // d, then Psi
  T* M = reinterpret_cast<T*>(scr + Ptot);          // m
  T* ZX = reinterpret_cast<T*>(scr + 2 * Ptot);     // zeta_x
  T* SX = reinterpret_cast<T*>(scr + 3 * Ptot);     // s_x
  T* DX = reinterpret_cast<T*>(scr + 4 * Ptot);     // d_x
  static_assert(sizeof(T) == sizeof(double), "8-byte plane elements");
  // (u, eta u)
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T uu = num<T>(u[o + j]), e = num<T>(eta[o + j]);
    b0[j] = mk(uu, e * uu);
  }
  __syncthreads();
  const cplx<T>* r = mr_deriv_pair<T>(b0, b1, P, kunit, tw);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    D[o + j] = r[j].x;
    M[o + j] = r[j].y;
  }
  __syncthreads();
  // (zeta, s)
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T e = num<T>(eta[o + j]), hh = num<T>(hgt[o + j]), g1 = num<T>(hx[o + j]);
    b0[j] = mk(e - hh, g1 * num<T>(u[o + j]));
  }
  __syncthreads();
  r = mr_deriv_pair<T>(b0, b1, P, kunit, tw);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    ZX[o + j] = r[j].x;
    SX[o + j] = r[j].y;
  }
  __syncthreads();
  // d -> d_x
  for (int j = threadIdx.x; j < n; j += kMrNT) b0[j] = mk(D[o + j], from_int<T>(0));
  __syncthreads();
  r = mr_deriv_pair<T>(b0, b1, P, kunit, tw);
  for (int j = threadIdx.x; j < n; j += kMrNT) DX[o + j] = r[j].x;
  __syncthreads();
  // Phi' -> Phi'_x; f_eta, and Psi kept for f_U
  const T third = num<T>(1.0 / 3.0);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T uu = num<T>(u[o + j]), e = num<T>(eta[o + j]), g1 = num<T>(hx[o + j]);
    const T d = D[o + j], m = M[o + j], s = g1 * uu;
    const T Q = uu * DX[o + j] - d * d, Sv = uu * SX[o + j];
    const T e2 = e * e;
    const T phi = e2 * e * Q * third + e2 * m * d + half(e2 * Sv) + e * m * s - e * uu * uu;
    const T psi = half(e2 * Q) + e * m * d + e * Sv + m * s;
    b0[j] = mk(phi, from_int<T>(0));
    D[o + j] = psi;                       // d is no longer needed
    f_eta[o + j] = -to_f64(m);
  }
  __syncthreads();
  r = mr_deriv_pair<T>(b0, b1, P, kunit, tw);
  const T gT = num<T>(g);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T e = num<T>(eta[o + j]), g1 = num<T>(hx[o + j]);
    f_U[o + j] = to_f64(r[j].x - gT * e * ZX[o + j] - g1 * D[o + j]);
  }
}

// ---- launchers (one launch over the generic instances ids[first, first + num)) ---------
MrArgs mr_args(const Layout1d& lay, int first) {
  MrArgs A;
  A.insts = lay.d_inst;
  A.ids = lay.d_ids + first;
  A.big = static_cast<cplx<double>*>(lay.mr_big);
  const long long len = lay.mr_tw_len;
  const char* base = static_cast<const char*>(lay.mr_tw);
  A.tw64 = reinterpret_cast<const cplx<double>*>(base);
  A.tw32 = reinterpret_cast<const cplx<float>*>(base + sizeof(cplx<double>) * len);
  A.twdf = reinterpret_cast<const cplx<df>*>(base + (sizeof(cplx<double>) + sizeof(cplx<float>)) * len);
  return A;
}

// Two transform buffers of the layout's largest generic n up to kMrSmemN, 16 bytes per
// entry.  The twiddle tables lie back to back (float64, float32, double-float; mr_tw_len
// entries each, an even count so that the double-float table starts on a 16-byte boundary).
size_t mr_smem(const Layout1d& lay) { return (size_t)2 * 16 * lay.mr_smem_n; }

template <typename K>
cudaError_t mr_attr(K k, size_t sm) {
  return raise_smem(k, sm);
}

}  // namespace

bool mr_in_smem(int n) { return n <= kMrSmemN; }

bool mr_size_ok(int n) {
  MrPlan P;
  return n >= 6 && n <= kMrMaxN && (n & (n - 1)) != 0 && mr_plan(n, P);
}

long long mr_twiddle_len(int n) { return n - 1; }

cudaError_t mr_twiddles_init(int n, long long off, const Layout1d& lay, cudaStream_t s) {
  const MrArgs A = mr_args(lay, 0);
  k_mr_twiddles<<<(n + 255) / 256, 256, 0, s>>>(
      n, const_cast<cplx<double>*>(A.tw64) + off, const_cast<cplx<float>*>(A.tw32) + off,
      const_cast<cplx<df>*>(A.twdf) + off);
  return cudaGetLastError();
}

cudaError_t mr_launch_deriv(const Layout1d& lay, int first, int num, const double* f,
                            double* fx, cudaStream_t s) {
  const size_t sm = mr_smem(lay);
  cudaError_t e = mr_attr(k_mr_deriv, sm);
  if (e) return e;
  k_mr_deriv<<<num, kMrNT, sm, s>>>(mr_args(lay, first), f, fx);
  return cudaGetLastError();
}

cudaError_t mr_launch_apply_G(const Layout1d& lay, int first, int num, const double* eta,
                              const double* hx, const double* u, double* Gu, cudaStream_t s) {
  const size_t sm = mr_smem(lay);
  cudaError_t e = mr_attr(k_mr_apply_G, sm);
  if (e) return e;
  k_mr_apply_G<<<num, kMrNT, sm, s>>>(mr_args(lay, first), eta, hx, u, Gu);
  return cudaGetLastError();
}

cudaError_t mr_launch_precond(const Layout1d& lay, int first, int num, const SolveRec* rec,
                              const double* r, double* z, cudaStream_t s) {
  const size_t sm = mr_smem(lay);
  cudaError_t e = mr_attr(k_mr_precond, sm);
  if (e) return e;
  k_mr_precond<<<num, kMrNT, sm, s>>>(mr_args(lay, first), rec, r, z);
  return cudaGetLastError();
}

cudaError_t mr_launch_pcg(const Layout1d& lay, int first, int num, int precision,
                          const double* eta, const double* hx, const double* b, double* x,
                          const SolveRec* given, int kind, double rtol, double rtol_inner,
                          int maxit, int max_refine, SolveRec* rec, void* ws, cudaStream_t s) {
  MrPcgArgs a;
  a.eta = eta;
  a.hx = hx;
  a.b = b;
  a.x = x;
  a.given = given;
  a.kind = kind;
  a.rtol = rtol;
  a.rtol_inner = rtol_inner;
  a.maxit = maxit;
  a.max_refine = max_refine;
  a.rec = rec;
  a.ws = static_cast<cplx<double>*>(ws);
  const size_t sm = mr_smem(lay);
  cudaError_t e;
  if (precision == SGN_PREC_MIXED) {
    if ((e = mr_attr(k_mr_pcg<true>, sm))) return e;
    k_mr_pcg<true><<<num, kMrNT, sm, s>>>(mr_args(lay, first), a);
  } else {
    if ((e = mr_attr(k_mr_pcg<false>, sm))) return e;
    k_mr_pcg<false><<<num, kMrNT, sm, s>>>(mr_args(lay, first), a);
  }
  return cudaGetLastError();
}

cudaError_t mr_launch_rhs(const Layout1d& lay, int first, int num, int precision, double g,
                          const double* eta, const double* u, const double* h,
                          const double* hx, double* f_eta, double* f_U, double* scratch,
                          cudaStream_t s) {
  const size_t sm = mr_smem(lay);
  cudaError_t e;
  if (precision == SGN_PREC_MIXED) {
    if ((e = mr_attr(k_mr_rhs<df>, sm))) return e;
    k_mr_rhs<df><<<num, kMrNT, sm, s>>>(mr_args(lay, first), g, eta, u, h, hx, f_eta, f_U,
                                       scratch, lay.points);
  } else {
    if ((e = mr_attr(k_mr_rhs<double>, sm))) return e;
    k_mr_rhs<double><<<num, kMrNT, sm, s>>>(mr_args(lay, first), g, eta, u, h, hx, f_eta, f_U,
                                           scratch, lay.points);
  }
  return cudaGetLastError();
}

}  // namespace sgn
