// Device helpers shared by the 1d kernel translation units (see sgn_1d.cu for the
// spectral-space formulation).
#pragma once
#include <type_traits>

#include "sgn_common.cuh"
#include "sgn_internal.h"

namespace sgn {
namespace d1 {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kLambdaPlus = 1.2675918792439982;    // (4 + sqrt 13)/6, Appendix A
constexpr double kLambdaMinus = 0.06574145408933513;  // (4 - sqrt 13)/6
constexpr double kFlatSlope = 1e-12;

__device__ __forceinline__ double mode_k(int m, int n, double kunit) {
  // m in [0, n/2]: k = kunit m, with the Nyquist wavenumber set to 0
  return (m == (n >> 1)) ? 0.0 : kunit * (double)m;
}

// ---------------------------------------------------------------------------------------
// a1: preconditioner coefficients by block reductions (Eq:FlatbathCoeff, Eq:Optcoeff,
// Eq:Optcoeffb, replacement remark of §4).  With CL = 2 the CTA holds one half of the
// instance (n points each) and the two halves' extrema meet through distributed shared
// memory; max and min are exact, so both CTAs form the same coefficients.
// ---------------------------------------------------------------------------------------
template <int NT, int CL = 1>
__device__ __forceinline__ void coeffs_block(const double* __restrict__ eta, const double* __restrict__ hx, int n,
                             int kind, double* red, SolveRec& R) {
  double emin = 1.0e308, emax = -1.0e308, g2max = 0.0, sopt = -1.0e308, bad = 0.0;
  for (int j = threadIdx.x; j < n; j += NT) {
    double e = eta[j], g = hx[j];
    double g2 = g * g;
    if (!(e > 0.0) || !(g2 < 1.0e300)) bad = 1.0;   // catches <= 0, NaN, Inf
    emin = fmin(emin, e);
    emax = fmax(emax, e);
    g2max = fmax(g2max, g2);
    sopt = fmax(sopt, e + kLambdaPlus * e * g2);
  }
  emin = block_min<NT>(emin, red);
  emax = block_max<NT>(emax, red);
  g2max = block_max<NT>(g2max, red);
  sopt = block_max<NT>(sopt, red);
  bad = block_max<NT>(bad, red);
  if constexpr (CL > 1) {
    __shared__ double xc[5];
    if (threadIdx.x == 0) {
      xc[0] = emin;
      xc[1] = emax;
      xc[2] = g2max;
      xc[3] = sopt;
      xc[4] = bad;
    }
    cluster_sync();
    const double* pc = peer(xc);
    emin = fmin(emin, pc[0]);
    emax = fmax(emax, pc[1]);
    g2max = fmax(g2max, pc[2]);
    sopt = fmax(sopt, pc[3]);
    bad = fmax(bad, pc[4]);
  }
  R.eta_min = emin;
  R.eta_max = emax;
  if (bad > 0.0) {
    R.status = SGN_ERR_NONPOSITIVE_DEPTH;
    R.sigma = R.alpha = R.kappa_ub = 0.0;
    R.flat = 0;
    return;
  }
  const double ratio3 = (emax / emin) * (emax / emin) * (emax / emin);
  const double smax = sqrt(g2max);
  R.flat = smax <= kFlatSlope;
  if (R.flat) {
    R.sigma = emax;
    R.alpha = emax * emax * emax / 3.0;
    R.kappa_ub = ratio3;
  } else if (kind == SGN_COEF_OPT) {
    R.sigma = sopt;
    R.alpha = kLambdaPlus * emax * emax * emax;
    R.kappa_ub = fmax(sopt / emin, (kLambdaPlus / kLambdaMinus) * ratio3);
  } else {
    R.sigma = emax * (1.0 + kLambdaPlus * g2max);
    R.alpha = kLambdaPlus * emax * emax * emax;
    R.kappa_ub = fmax((emax / emin) * (1.0 + kLambdaPlus * g2max),
                      (kLambdaPlus / kLambdaMinus) * ratio3);
  }
  R.status = SGN_OK;
}

// ---------------------------------------------------------------------------------------
// Spectral constants of one instance in the working precision T, so that per-mode work
// never leaves T (on this part one stray float64 op costs ~62 float32 ops).
// ---------------------------------------------------------------------------------------
template <typename T>
struct Spec {
  T kunit;     // 2 pi / L
  T sigma;     // preconditioner A = sigma I - alpha d^2/dx^2
  T alpha;
  int n, h;
  __device__ __forceinline__ T k(int m) const {        // m in [0, n/2], Nyquist -> 0
    return m == h ? from_int<T>(0) : kunit * from_int<T>(m);
  }
  __device__ __forceinline__ T weight(int m) const {   // Parseval weight on half spectra
    return (m == 0 || m == h) ? from_int<T>(1) : from_int<T>(2);
  }
};

template <typename T>
__device__ __forceinline__ Spec<T> make_spec(int n, double L, double sigma, double alpha) {
  Spec<T> s;
  s.kunit = num<T>(2.0 * kPi / L);
  s.sigma = num<T>(sigma);
  s.alpha = num<T>(alpha);
  s.n = n;
  s.h = n >> 1;
  return s;
}

// ---------------------------------------------------------------------------------------
// Matvec in spectral form.  `get(m)` returns the half-spectrum coefficient of the input
// for m in [0, n/2] (it may read buf[m]: each thread writes only buf[m] and buf[n-m] of
// the modes it read).  On return buf holds Y = FFT(w + i q); extract (G v)_m with gv_mode.
// ---------------------------------------------------------------------------------------
// Inverse FFT of Z (already in buf), pointwise coefficients, forward FFT.
// With wsub set, w - wsub is transformed instead of w, so the result is (G v - wsub)^.
// With vxout set, the input's derivative v_x (the imaginary part of the packed inverse) is
// stored there too, in T.
template <typename T, int NT, int MAXB, typename Coef>
__device__ __forceinline__ void matvec_core(cplx<T>* buf, int n, int log2n, const Coef& coef,
                                            double* __restrict__ vout,
                                            const cplx<T>* __restrict__ tw,
                                            const double* __restrict__ wsub = nullptr,
                                            T* __restrict__ vxout = nullptr) {
  cta_fft<T, NT, MAXB>(buf, n, log2n, true, tw);
  const T inv_n = num<T>(1.0 / (double)n);
  for (int j = threadIdx.x; j < n; j += NT) {
    cplx<T> z = buf[j];
    T v = z.x * inv_n, vx = z.y * inv_n;
    T c1, c2, c3;
    coef(j, c1, c2, c3);
    if (vout) vout[j] = to_f64(v);
    if (vxout) vxout[j] = vx;
    T w = c1 * v + c2 * vx;
    if (wsub) w = w - num<T>(wsub[j]);
    buf[j] = mk(w, c2 * v + c3 * vx);
  }
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, log2n, false, tw);
}

template <typename T, int NT, int MAXB, typename Get, typename Coef>
__device__ __forceinline__ void spectral_matvec(cplx<T>* buf, const Spec<T>& sp, int log2n,
                                                Get get, Coef coef, double* __restrict__ vout,
                                                const cplx<T>* __restrict__ tw,
                                                const double* __restrict__ wsub = nullptr,
                                                T* __restrict__ vxout = nullptr) {
  const int n = sp.n, h = sp.h;
  const T one = from_int<T>(1);
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<T> v = get(m);
    // the DC and Nyquist coefficients of a real field are real: drop rounding residue
    if (m == 0 || m == h) v = mk(v.x, from_int<T>(0));
    const T k = sp.k(m);
    buf[m] = v * (one - k);
    if (m > 0 && m < h) buf[n - m] = conj(v) * (one + k);
  }
  __syncthreads();
  matvec_core<T, NT, MAXB>(buf, n, log2n, coef, vout, tw, wsub, vxout);
}

// (G v)_m = w_m - i k_m q_m = ((1 - k) Y_m + (1 + k) conj(Y_{n-m})) / 2
template <typename T>
__device__ __forceinline__ cplx<T> gv_mode(const cplx<T>* buf, int m, int n, T k) {
  const T one = from_int<T>(1);
  cplx<T> y = buf[m];
  cplx<T> yc = conj(buf[(n - m) & (n - 1)]);
  cplx<T> s = y * (one - k) + yc * (one + k);
  return mk(half(s.x), half(s.y));
}

// float64 coefficients of Def:MatrixM (1d) computed from eta and h_x on the fly
struct CoefGlobal64 {
  const double* eta;
  const double* hx;
  __device__ __forceinline__ void operator()(int j, double& c1, double& c2, double& c3) const {
    double e = eta[j], g = hx[j];
    c1 = e * (1.0 + g * g);
    c2 = 0.5 * e * e * g;
    c3 = e * e * e * (1.0 / 3.0);
  }
};

// float32 coefficients: c1 = eta (1 + h_x^2), c2 = eta^2 h_x / 2, c3 = eta^3 / 3 in smem
struct CoefSmem32 {
  const float* c;     // [3][n]
  int n;
  __device__ __forceinline__ void operator()(int j, float& c1, float& c2, float& c3) const {
    c1 = c[j];
    c2 = c[n + j];
    c3 = c[2 * n + j];
  }
};

// double-float coefficients: the float32 parts in smem, the remainders in global memory
struct CoefDF {
  const float* hi;    // [3][n] shared
  const float* lo;    // [3][n] global
  int n;
  __device__ __forceinline__ void operator()(int j, df& c1, df& c2, df& c3) const {
    c1 = df(hi[j], lo[j]);
    c2 = df(hi[n + j], lo[n + j]);
    c3 = df(hi[2 * n + j], lo[2 * n + j]);
  }
};

// Splits the float64 coefficients into float32 parts (smem) and remainders (global).
template <int NT>
__device__ __forceinline__ void split_coefficients(const double* __restrict__ eta,
                                                   const double* __restrict__ hx, int n,
                                                   float* __restrict__ c_hi,
                                                   float* __restrict__ c_lo) {
  for (int j = threadIdx.x; j < n; j += NT) {
    double e = eta[j], g = hx[j];
    double c[3] = {e * (1.0 + g * g), 0.5 * e * e * g, e * e * e * (1.0 / 3.0)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float hi = (float)c[q];
      c_hi[q * n + j] = hi;
      if (c_lo) c_lo[q * n + j] = (float)(c[q] - (double)hi);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Derivative pair: buf <- load(j) = f + i g, forward FFT, times i k_m (Nyquist 0) / n,
// inverse FFT; on return buf[j] = f_x + i g_x (D is real, so it acts on both parts).
// ---------------------------------------------------------------------------------------
template <typename T, int NT, int MAXB, typename Load>
__device__ __forceinline__ void deriv_pair(cplx<T>* buf, int n, int log2n, T kunit_over_n,
                                           Load load, const cplx<T>* __restrict__ tw) {
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = load(j);
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, log2n, false, tw);
  for (int m = threadIdx.x; m < n; m += NT) {
    T k = kunit_over_n * from_int<T>(wave_index(m, n));
    buf[m] = mul_pi(buf[m]) * k;
  }
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, log2n, true, tw);
}

// ---------------------------------------------------------------------------------------
// Size classes (one per log2 n).
// ---------------------------------------------------------------------------------------
template <int V>
using IC = std::integral_constant<int, V>;

// One launch per size class.  When a layout holds several classes they run concurrently on
// the layout's side streams (event fork from `s`, join back into `s`; largest class first),
// so a class that occupies few SMs does not leave the rest of the GPU idle.
// call(l, first, num, stream) launches class l = log2 n (kGenericClass: the sizes that are
// not powers of two).
template <typename Call>
cudaError_t fan_classes(const Layout1d& lay, cudaStream_t s, Call&& call) {
  int ncls = 0;
  for (int i = 0; i < kNumClassSlots; ++i) {
    const int l = class_at(i);
    ncls += lay.class_end[l] > lay.class_begin[l];
  }
  const bool fan = ncls > 1 && lay.side[0] != nullptr;
  if (fan && cudaEventRecord(lay.fork, s) != cudaSuccess) return cudaGetLastError();
  int ci = 0;
  for (int i = 0; i < kNumClassSlots; ++i) {
    const int l = class_at(i);
    const int b = lay.class_begin[l], e = lay.class_end[l];
    if (e <= b) continue;
    cudaStream_t cs = s;
    if (fan) {
      cs = lay.side[ci];
      if (cudaStreamWaitEvent(cs, lay.fork, 0) != cudaSuccess) return cudaGetLastError();
    }
    const cudaError_t err = call(l, b, e - b, cs);
    if (err != cudaSuccess) return err;
    if (fan) {
      if (cudaEventRecord(lay.join[ci], cs) != cudaSuccess ||
          cudaStreamWaitEvent(s, lay.join[ci], 0) != cudaSuccess)
        return cudaGetLastError();
    }
    ++ci;
  }
  return cudaSuccess;
}

// The generic class's launch of an operation that has no generic kernel (the API rejects
// such layouts first).
struct NoGeneric {
  cudaError_t operator()(int, int, cudaStream_t) const { return cudaErrorNotSupported; }
};

// Size-class dispatch for the cta_fft kernels: NT = clamp(n/8, 32, 512) threads, MAXB =
// n/(4 NT) butterflies per thread per radix-4 stage (n = 16384: 1024 threads, and the
// transform buffer in the layout's global scratch instead of shared memory).  gen(first,
// num, stream) launches the generic class.
template <typename Fn, typename Gen = NoGeneric>
cudaError_t for_each_class(const Layout1d& lay, cudaStream_t s, Fn&& fn, Gen&& gen = Gen{}) {
  return fan_classes(lay, s, [&](int l, int b, int num, cudaStream_t cs) -> cudaError_t {
    switch (l) {
      case kGenericClass: return gen(b, num, cs);
      case 3: case 4: case 5: case 6: case 7: return fn(IC<32>{}, IC<1>{}, l, b, num, cs);
      case 8: return fn(IC<32>{}, IC<2>{}, l, b, num, cs);
      case 9: return fn(IC<64>{}, IC<2>{}, l, b, num, cs);
      case 10: return fn(IC<128>{}, IC<2>{}, l, b, num, cs);
      case 11: return fn(IC<256>{}, IC<2>{}, l, b, num, cs);
      case 12: return fn(IC<512>{}, IC<2>{}, l, b, num, cs);
      case 13: return fn(IC<512>{}, IC<4>{}, l, b, num, cs);
      case 14: return fn(IC<1024>{}, IC<4>{}, l, b, num, cs);
      default: return cudaErrorInvalidValue;
    }
  });
}

// Size-class dispatch for the register-FFT kernels, templated on log2 n; gen as above.
template <typename Fn, typename Gen = NoGeneric>
cudaError_t for_each_size(const Layout1d& lay, cudaStream_t s, Fn&& fn, Gen&& gen = Gen{}) {
  return fan_classes(lay, s, [&](int l, int b, int num, cudaStream_t cs) -> cudaError_t {
    switch (l) {
      case kGenericClass: return gen(b, num, cs);
      case 3: return fn(IC<3>{}, b, num, cs);
      case 4: return fn(IC<4>{}, b, num, cs);
      case 5: return fn(IC<5>{}, b, num, cs);
      case 6: return fn(IC<6>{}, b, num, cs);
      case 7: return fn(IC<7>{}, b, num, cs);
      case 8: return fn(IC<8>{}, b, num, cs);
      case 9: return fn(IC<9>{}, b, num, cs);
      case 10: return fn(IC<10>{}, b, num, cs);
      case 11: return fn(IC<11>{}, b, num, cs);
      case 12: return fn(IC<12>{}, b, num, cs);
      case 13: return fn(IC<13>{}, b, num, cs);
      case 14: return fn(IC<14>{}, b, num, cs);
      default: return cudaErrorInvalidValue;
    }
  });
}

// num instances of CL CTAs each (CL = 2: thread-block clusters of two consecutive CTAs)
template <int CL, typename... P>
cudaError_t launch_clustered(void (*kernel)(P...), int num, int threads, size_t smem,
                             cudaStream_t s, const P&... args) {
  if constexpr (CL == 1) {
    kernel<<<num, threads, smem, s>>>(args...);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(num * CL), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
  }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return raise_smem(kernel, bytes);
}

}  // namespace d1
}  // namespace sgn
