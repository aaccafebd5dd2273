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
// Eq:Optcoeffb, replacement remark of §4).
// ---------------------------------------------------------------------------------------
template <int NT>
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
// Matvec in spectral form.  `get(m)` returns the half-spectrum coefficient of the input
// for m in [0, n/2] (it may read buf[m]: each thread writes only buf[m] and buf[n-m] of
// the modes it read).  On return buf holds Y = FFT(w + i q); extract (G v)_m with gv_mode.
// ---------------------------------------------------------------------------------------
template <typename T, int NT, int MAXB, typename Get, typename Coef>
__device__ __forceinline__ void spectral_matvec(cplx<T>* buf, int n, int log2n, double kunit,
                                                Get get, Coef coef, double* __restrict__ vout,
                                                const cplx<T>* __restrict__ tw) {
  const int h = n >> 1;
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<T> v = get(m);
    T k = (T)mode_k(m, n, kunit);
    buf[m] = v * ((T)1 - k);
    if (m > 0 && m < h) buf[n - m] = conj(v) * ((T)1 + k);
  }
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, log2n, true, tw);
  const T inv_n = (T)1 / (T)n;
  for (int j = threadIdx.x; j < n; j += NT) {
    cplx<T> z = buf[j];
    T v = z.x * inv_n, vx = z.y * inv_n;
    T c1, c2, c3;
    coef(j, c1, c2, c3);
    if (vout) vout[j] = (double)v;
    buf[j] = mk(c1 * v + c2 * vx, c2 * v + c3 * vx);
  }
  __syncthreads();
  cta_fft<T, NT, MAXB>(buf, n, log2n, false, tw);
}

template <typename T>
__device__ __forceinline__ cplx<T> gv_mode(const cplx<T>* buf, int m, int n, T k) {
  cplx<T> y = buf[m];
  cplx<T> yc = conj(buf[(n - m) & (n - 1)]);
  return (y * ((T)1 - k) + yc * ((T)1 + k)) * (T)0.5;
}

// FP64 coefficients of Def:MatrixM (1d) computed from eta and h_x on the fly
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

struct CoefSmem32 {
  const float* c;     // [3][n]
  int n;
  __device__ __forceinline__ void operator()(int j, float& c1, float& c2, float& c3) const {
    c1 = c[j];
    c2 = c[n + j];
    c3 = c[2 * n + j];
  }
};

// ---------------------------------------------------------------------------------------
// a7: right-hand side f(w, p) of Eq:DAE_DSWE with F from Def:bigF, float64.
// ---------------------------------------------------------------------------------------
template <int NT, int MAXB, typename Load>
__device__ __forceinline__ void deriv_pair(cplx<double>* buf, int n, int log2n, double kunit,
                                           Load load, const cplx<double>* __restrict__ tw) {
  for (int j = threadIdx.x; j < n; j += NT) buf[j] = load(j);
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, log2n, false, tw);
  const double inv_n = 1.0 / n;
  for (int m = threadIdx.x; m < n; m += NT) {
    double k = kunit * (double)wave_index(m, n) * inv_n;
    buf[m] = mul_pi(buf[m]) * k;
  }
  __syncthreads();
  cta_fft<double, NT, MAXB>(buf, n, log2n, true, tw);
}

// ---------------------------------------------------------------------------------------
// Size-class dispatch: NT = clamp(n/8, 32, 512) threads, MAXB = n/(4 NT) butterflies
// per thread per radix-4 stage.
// ---------------------------------------------------------------------------------------
template <int V>
using IC = std::integral_constant<int, V>;

template <typename Fn>
cudaError_t for_each_class(const Layout1d& lay, Fn&& fn) {
  for (int l = 3; l <= 13; ++l) {
    const int b = lay.class_begin[l], e = lay.class_end[l];
    if (e <= b) continue;
    cudaError_t err = cudaSuccess;
    switch (l) {
      case 3: case 4: case 5: case 6: case 7: err = fn(IC<32>{}, IC<1>{}, l, b, e - b); break;
      case 8: err = fn(IC<32>{}, IC<2>{}, l, b, e - b); break;
      case 9: err = fn(IC<64>{}, IC<2>{}, l, b, e - b); break;
      case 10: err = fn(IC<128>{}, IC<2>{}, l, b, e - b); break;
      case 11: err = fn(IC<256>{}, IC<2>{}, l, b, e - b); break;
      case 12: err = fn(IC<512>{}, IC<2>{}, l, b, e - b); break;
      case 13: err = fn(IC<512>{}, IC<4>{}, l, b, e - b); break;
      default: return cudaErrorInvalidValue;
    }
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace d1
}  // namespace sgn
