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

namespace sgn {
namespace {

using d1::kPi;
constexpr int kMrNT = 256;
constexpr int kMrMaxN = 16384;       // largest generic n
constexpr int kMrSmemN = 6144;       // largest n whose two transform buffers (192 KB) are in
                                     // shared memory; above it they are in global memory
constexpr int kMrMaxStages = 16;

// ---- plan: radices in order (8 ... 8, then 4 or 2, then 5 ... 5, then 3 ... 3) ------------
struct MrPlan {
  int n, ns;
  int n8, r42, n5;       // radix-8 stages, the 4 or 2 stage (0: none), radix-5 stages
  __host__ __device__ int radix(int st) const {
    if (st < n8) return 8;
    st -= n8;
    if (r42) {
      if (st == 0) return r42;
      --st;
    }
    return st < n5 ? 5 : 3;
  }
};

__host__ __device__ inline bool mr_plan(int n, MrPlan& P) {
  int a = 0, b = 0, c = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  while (m % 5 == 0) { m /= 5; ++c; }
  if (m != 1 || a < 1) return false;
  P.n = n;
  P.n8 = a / 3;
  P.r42 = a % 3 == 2 ? 4 : (a % 3 == 1 ? 2 : 0);
  P.n5 = c;
  P.ns = P.n8 + (P.r42 != 0) + c + b;
  return P.ns <= kMrMaxStages;
}

// ---- small DFTs in registers, natural order --------------------------------------------
template <typename T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> a, bool inv) {   // * (-+i)
  return inv ? mul_pi(a) : mul_mi(a);
}

template <typename T, int R>
__device__ __forceinline__ void mr_dft(cplx<T>* x, bool inv) {
  if constexpr (R == 2) {
    const cplx<T> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else if constexpr (R == 4) {
    const cplx<T> s02 = x[0] + x[2], d02 = x[0] - x[2], s13 = x[1] + x[3], d13 = x[1] - x[3];
    const cplx<T> r13 = mul_i(d13, inv);
    x[0] = s02 + s13;
    x[1] = d02 + r13;
    x[2] = s02 - s13;
    x[3] = d02 - r13;
  } else if constexpr (R == 3) {
    // y1,2 = x0 - (x1 + x2)/2 -+ i (sqrt3/2)(x1 - x2)
    const T h3 = num<T>(0.86602540378443864676);
    const cplx<T> s = x[1] + x[2], d = x[1] - x[2];
    const cplx<T> m = x[0] - mk(half(s.x), half(s.y));
    const cplx<T> t = mul_i(d, inv) * h3;
    x[0] = x[0] + s;
    x[1] = m + t;
    x[2] = m - t;
  } else if constexpr (R == 5) {
    // y_s = sum_r x_r w^{r s}, w = e^{-+2 pi i / 5}, pairing r and 5 - r
    const T c1 = num<T>(0.30901699437494742410), c2 = num<T>(-0.80901699437494742410);
    const T s1 = num<T>(0.95105651629515357212), s2 = num<T>(0.58778525229247312917);
    const cplx<T> a1 = x[1] + x[4], b1 = x[1] - x[4], a2 = x[2] + x[3], b2 = x[2] - x[3];
    const cplx<T> m1 = x[0] + a1 * c1 + a2 * c2, m2 = x[0] + a1 * c2 + a2 * c1;
    // -+i (s1 b1 + s2 b2) and -+i (s2 b1 - s1 b2)
    const cplx<T> t1 = mul_i(b1 * s1 + b2 * s2, inv), t2 = mul_i(b1 * s2 - b2 * s1, inv);
    x[0] = x[0] + a1 + a2;
    x[1] = m1 + t1;
    x[4] = m1 - t1;
    x[2] = m2 + t2;
    x[3] = m2 - t2;
  } else {
    // 8 = 2 x 4
    cplx<T> e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    mr_dft<T, 4>(e, inv);
    mr_dft<T, 4>(o, inv);
    const T r = num<T>(0.70710678118654752440);
    const cplx<T> o1 = o[1], o3 = o[3];
    const cplx<T> w1 = inv ? mk((o1.x - o1.y) * r, (o1.x + o1.y) * r)
                           : mk((o1.x + o1.y) * r, (o1.y - o1.x) * r);
    const cplx<T> w2 = mul_i(o[2], inv);
    const cplx<T> w3 = inv ? mk(-(o3.x + o3.y) * r, (o3.x - o3.y) * r)
                           : mk((o3.y - o3.x) * r, -(o3.x + o3.y) * r);
    x[0] = e[0] + o[0];
    x[4] = e[0] - o[0];
    x[1] = e[1] + w1;
    x[5] = e[1] - w1;
    x[2] = e[2] + w2;
    x[6] = e[2] - w2;
    x[3] = e[3] + w3;
    x[7] = e[3] - w3;
  }
}

// One radix-R Stockham stage at sub-length p: butterfly i reads src[i + r n/R], twiddles by
// w^{r k} (k = i mod p, table block at p - 1: entry (r - 1) p + k), writes output s to
// dst[(i - k) R + k + s p].
template <typename T, int R>
__device__ __forceinline__ void mr_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                         int n, int p, bool inv, const cplx<T>* __restrict__ tw) {
  const int q = n / R;
  for (int i = threadIdx.x; i < q; i += kMrNT) {
    const int k = i % p;
    cplx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = src[i + r * q];
    if (p > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul_tw(x[r], tw[p - 1 + (r - 1) * p + k], inv);
    }
    mr_dft<T, R>(x, inv);
    const int o = (i - k) * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) dst[o + s * p] = x[s];
  }
  __syncthreads();
}

// The transform of a (length n, natural order) with b as the other buffer; returns the
// buffer holding the result.  Forward: X_m = sum_j x_j e^{-2 pi i j m / n}; inverse without
// the 1/n.  Callers synchronise before it; it returns after a barrier.
template <typename T>
__device__ cplx<T>* mr_fft(cplx<T>* a, cplx<T>* b, const MrPlan& P, bool inv,
                           const cplx<T>* tw) {
  cplx<T>* src = a;
  cplx<T>* dst = b;
  int p = 1;
  for (int st = 0; st < P.ns; ++st) {
    const int R = P.radix(st);
    if (R == 8) mr_stage<T, 8>(src, dst, P.n, p, inv, tw);
    else if (R == 4) mr_stage<T, 4>(src, dst, P.n, p, inv, tw);
    else if (R == 2) mr_stage<T, 2>(src, dst, P.n, p, inv, tw);
    else if (R == 5) mr_stage<T, 5>(src, dst, P.n, p, inv, tw);
    else mr_stage<T, 3>(src, dst, P.n, p, inv, tw);
    p *= R;
    cplx<T>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

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
  cplx<T>* F = mr_fft<T>(A, B, P, false, tw);
  const double inv_n = 1.0 / n;
  for (int m = threadIdx.x; m < n; m += kMrNT) F[m] = mul_pi(F[m]) * num<T>(kunit * wave_index(m, n) * inv_n);
  __syncthreads();
  return mr_fft<T>(F, F == A ? B : A, P, true, tw);
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
  cplx<T>* z = mr_fft<T>(a, b, P, true, tw);
  const T inv_n = num<T>(1.0 / n);
  for (int j = threadIdx.x; j < n; j += kMrNT) {
    const T v = z[j].x * inv_n, vx = z[j].y * inv_n;
    T c1, c2, c3;
    coef(j, c1, c2, c3);
    z[j] = mk(c1 * v + c2 * vx, c2 * v + c3 * vx);
  }
  __syncthreads();
  cplx<T>* Y = mr_fft<T>(z, z == a ? b : a, P, false, tw);
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
  cplx<double>* V = mr_fft<double>(a, b, P, false, tw);
  cplx<double>* o = V == a ? b : a;
  // (G u)^ of modes 0..n/2 into V itself: mode m is read and written only by the thread
  // that computes it (its mirror n - m is above n/2 and never written)
  mr_matvec<double>(V, o, P, kunit, tw, Coef64{eta + I.off, hx + I.off}, V);
  // V[0..h] = (G u)^; build the Hermitian full spectrum and invert
  for (int m = threadIdx.x; m < h; m += kMrNT)
    if (m > 0) V[n - m] = conj(V[m]);
  __syncthreads();
  const cplx<double>* x = mr_fft<double>(V, o, P, true, tw);
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
  cplx<double>* F = mr_fft<double>(a, b, P, false, tw);
  for (int m = threadIdx.x; m < n; m += kMrNT) {
    const double k = kunit * wave_index(m, n);
    F[m] = F[m] * (1.0 / ((sigma + alpha * k * k) * (double)n));
  }
  __syncthreads();
  const cplx<double>* x = mr_fft<double>(F, F == a ? b : a, P, true, tw);
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
  cplx<double>* Y = mr_fft<double>(d0, d1, P, false, tws.d);
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
    const cplx<double>* x = mr_fft<double>(d0, d1, P, true, tws.d);
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
    const cplx<df>* x = mr_fft<df>(h0, h1, P, true, tws.h);
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

// e^{-2 pi i r k / (p R)} of every stage of n's plan, in float64, float32 and double-float
__global__ void k_mr_twiddles(int n, cplx<double>* t64, cplx<float>* t32, cplx<df>* tdf) {
  MrPlan P;
  mr_plan(n, P);
  int p = 1;
  for (int st = 0; st < P.ns; ++st) {
    const int R = P.radix(st);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (R - 1) * p;
         e += gridDim.x * blockDim.x) {
      const int r = 1 + e / p, k = e - (r - 1) * p;
      // the angle -2 r k / (p R) in units of pi, reduced exactly: (r k mod pR) / (pR)
      const long long num_ = (long long)r * k % ((long long)p * R);
      double sn, cs;
      sincospi(-2.0 * (double)num_ / (double)(p * R), &sn, &cs);
      t64[p - 1 + e] = mk(cs, sn);
      t32[p - 1 + e] = mk((float)cs, (float)sn);
      tdf[p - 1 + e] = mk(df(cs), df(sn));
    }
    p *= R;
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

// two transform buffers of the layout's largest generic n up to kMrSmemN, 16 bytes per entry.  The tables
// lie back to back (float64, float32, double-float; mr_tw_len entries each, an even count
// so that the double-float table starts on a 16-byte boundary).
size_t mr_smem(const Layout1d& lay) { return (size_t)2 * 16 * lay.mr_smem_n; }

template <typename K>
cudaError_t mr_attr(K k, size_t sm) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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
