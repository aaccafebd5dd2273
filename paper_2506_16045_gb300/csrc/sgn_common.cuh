// Device building blocks shared by the SGN kernels: complex arithmetic, the twiddle
// table, an in-shared-memory Stockham FFT run by one CTA, and deterministic block
// reductions with FP64 accumulation.
//
// Spectral convention (§6.1 of the paper): forward transform X_m = sum_j x_j e^{-2 pi i jm/n},
// inverse without the 1/n factor (callers scale); wavenumber k_m = 2 pi m / L for
// m < n/2, k_m = 2 pi (m - n) / L for m > n/2, and k_{n/2} = 0.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sgn_internal.h"

namespace sgn {

// Raises a kernel's dynamic shared-memory limit to the most the device allows it (the opt-in
// maximum less the kernel's static shared memory) when a launch needs more than the default
// 48 KB.  Every caller writes the same value for a kernel, so layouts of different sizes
// (and threads) never lower the limit under one another's launches: a limit set to each
// layout's own size let a smaller layout's setting make a larger layout's later launch fail.
template <typename K>
cudaError_t raise_smem(K kernel, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e) return e;
  if (fa.sharedSizeBytes + bytes <= 48 * 1024) return cudaSuccess;   // the default limit
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)))
    return e;
  const long long lim = (long long)optin - (long long)fa.sharedSizeBytes;
  if (lim < (long long)bytes) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

// -------------------------------------------------------------------------------------
// Double-float number: value = hi + lo with |lo| <= ulp(hi)/2, ~48-bit significand, built
// from float32 operations only (error-free transformations: Knuth's two-sum and the
// fused-multiply-add two-product, as in Dekker (1971) and the QD library of Hida, Li and
// Bailey).  On this part float64 FMA throughput is 1/62 of float32; a double-float add
// costs 11 float32 operations and a multiply 7, so float64-grade transforms run several
// times faster in this form.
// -------------------------------------------------------------------------------------
// Conversions between float64 and float32 / double-float done with integer and float32
// operations only: on this part every float64 instruction, conversions included, runs at
// 1/62 of the float32 rate.
//
// f64 -> double-float: hi takes the top 24 significand bits, lo the next 29 rounded to 24,
// then one fast two-sum renormalises (|lo| <= ulp(hi)/2); relative error <= 2^-48.  Values
// below 2^-74 in magnitude keep only hi (absolute error < 2^-98), values below 2^-126 become
// zero, and values beyond the float32 range take the float64 conversion.
struct df;
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
  const long long b = __double_as_longlong(d);
  const int h32 = (int)(b >> 32);
  const int e = (h32 >> 20) & 0x7ff;
  const unsigned sign = (unsigned)h32 & 0x80000000u;
  const unsigned top = (unsigned)((b >> 29) & 0x7fffff);
  if (e >= 949 && e <= 1150) {
    const float h = __int_as_float((int)(sign | ((unsigned)(e - 896) << 23) | top));
    const float r = __int2float_rn((int)(b & 0x1fffffff)) * __int_as_float((e - 948) << 23);
    const float l = sign ? -r : r;
    const float s = __fadd_rn(h, l);
    hi = s;
    lo = __fsub_rn(l, __fsub_rn(s, h));
  } else if (e > 1150) {
    hi = __double2float_rn(d);
    lo = 0.0f;
  } else {
    hi = (e >= 897) ? __int_as_float((int)(sign | ((unsigned)(e - 896) << 23) | top)) : 0.0f;
    lo = 0.0f;
  }
}
// exact float32 -> float64 (zero for float32 subnormals, which only low parts can be)
__device__ __forceinline__ double f64_of(float f) {
  const int fb = __float_as_int(f);
  const int ef = (fb >> 23) & 0xff;
  if (ef == 0) return 0.0;
  if (ef == 255) return (double)f;
  return __longlong_as_double(((long long)(fb & 0x80000000) << 32) |
                              ((long long)(ef + 896) << 52) | ((long long)(fb & 0x7fffff) << 29));
}

struct df {
  float hi, lo;
  __host__ __device__ df() {}
  __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df(double d) { split_f64(d, hi, lo); }
  __device__ __forceinline__ explicit df(int i) : hi((float)i), lo(0.0f) {}   // |i| < 2^24
  __device__ __forceinline__ explicit operator double() const { return f64_of(hi) + f64_of(lo); }
};

// The _rn intrinsics are never contracted into FMAs, which the error-free transformations
// rely on (each rounding must be the plain rounding of one operation).
__device__ __forceinline__ df operator+(df a, df b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float h = __fadd_rn(s, e);
  return df(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float h = __fadd_rn(p, e);
  return df(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// Conversions used by the generic kernels: num<T>(double), from_int<T>(int), to_f64(T).
template <typename T>
__device__ __forceinline__ T num(double d) { return (T)d; }
template <>
__device__ __forceinline__ df num<df>(double d) { return df(d); }
template <typename T>
__device__ __forceinline__ T from_int(int m) { return (T)m; }
template <>
__device__ __forceinline__ df from_int<df>(int m) { return df((float)m, 0.0f); }  // |m| < 2^24
__device__ __forceinline__ df half(df a) { return df(a.hi * 0.5f, a.lo * 0.5f); }
__device__ __forceinline__ float half(float a) { return a * 0.5f; }
__device__ __forceinline__ double half(double a) { return a * 0.5; }
// reciprocal in the working precision (float: correctly rounded, no float64 involved)
__device__ __forceinline__ float recip(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(df v) { return f64_of(v.hi) + f64_of(v.lo); }
// leading float32 part (for float32 estimates such as residual norms)
__device__ __forceinline__ float lead(float v) { return v; }
__device__ __forceinline__ float lead(double v) { return (float)v; }
__device__ __forceinline__ float lead(df v) { return v.hi; }

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b) when conj_b, else a * b (used for forward/inverse twiddles from one table)
template <typename T>
__device__ __forceinline__ cplx<T> cmul_tw(cplx<T> a, cplx<T> w, bool inverse) {
  T wy = inverse ? -w.y : w.y;
  return mk(a.x * w.x - a.y * wy, a.x * wy + a.y * w.x);
}
template <typename T>
__device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.x, -a.y); }
// multiply by i (inverse=false -> -i for the forward 4-point kernel's sign)
template <typename T>
__device__ __forceinline__ cplx<T> mul_pi(cplx<T> a) { return mk(-a.y, a.x); }   // * (+i)
template <typename T>
__device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) { return mk(a.y, -a.x); }   // * (-i)

// e^{-+2 pi i j / m} for integers j and m = 2^log2m, float32, computed in registers
// (sincospif of the exactly representable argument 2j/m) instead of a table load.
__device__ __forceinline__ cplx<float> twiddle_f32(int j, int log2m, bool inverse) {
  float s, c;
  sincospif(__int_as_float((128 - log2m) << 23) * (float)j, &s, &c);   // (2/m) j
  return mk(c, inverse ? s : -s);
}

// Signed integer wavenumber index of mode m for length n, with the n/2 mode mapped to 0.
__device__ __forceinline__ int wave_index(int m, int n) {
  int h = n >> 1;
  return m < h ? m : (m == h ? 0 : m - n);
}

// -------------------------------------------------------------------------------------
// In-shared-memory complex FFT (Stockham autosort, one radix-2 stage when log2 n is odd,
// then radix-4 stages).  Stage with current sub-transform length p: butterfly i takes the
// R inputs buf[i + r n/R], twiddles them by w^{r k}, w = e^{-+2 pi i/(p R)}, k = i mod p,
// and writes the R outputs to ((i - k) R + k) + s p.  Each thread keeps its butterflies'
// outputs in registers between a barrier after all reads and the writes, so the transform
// is in place.  MAXB bounds butterflies per thread per radix-4 stage: n/4 <= MAXB*NT.
// All NT threads must call; returns after a barrier.
// -------------------------------------------------------------------------------------
// Twiddles come from `tw` (a table of e^{-2 pi i j / 2^14}); with tw == nullptr (float32
// only) they are computed in registers, which avoids L2 round trips when shared memory
// leaves little L1 for the table.
template <typename T, int NT, int MAXB>
__device__ __forceinline__ void cta_fft(cplx<T>* buf, int n, int log2n, bool inverse,
                                        const cplx<T>* __restrict__ tw) {
  const int t = threadIdx.x;
  int p = 1;
  int lp = 0;                                    // log2 p
  if (log2n & 1) {
    const int h = n >> 1;
    cplx<T> y0[2 * MAXB], y1[2 * MAXB];
    int dst[2 * MAXB];
#pragma unroll
    for (int b = 0; b < 2 * MAXB; ++b) {
      int i = t + b * NT;
      if (i < h) {
        cplx<T> a0 = buf[i];
        cplx<T> a1 = buf[i + h];
        // p = 1 here: k = 0, no twiddle
        y0[b] = a0 + a1;
        y1[b] = a0 - a1;
        dst[b] = i * 2;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 2 * MAXB; ++b) {
      int i = t + b * NT;
      if (i < h) {
        buf[dst[b]] = y0[b];
        buf[dst[b] + 1] = y1[b];
      }
    }
    __syncthreads();
    p = 2;
    lp = 1;
  }
  const int q = n >> 2;
  while (p < n) {
    cplx<T> y[MAXB][4];
    int dst[MAXB];
    const int tshift = kTwiddleLog2 - lp - 2;    // table stride NMAX/(4p) as a shift
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      int i = t + b * NT;
      if (i < q) {
        int k = i & (p - 1);
        cplx<T> a0 = buf[i];
        cplx<T> a1 = buf[i + q];
        cplx<T> a2 = buf[i + 2 * q];
        cplx<T> a3 = buf[i + 3 * q];
        if (p > 1) {
          if constexpr (std::is_same<T, float>::value) {
            if (tw == nullptr) {
              // w = e^{-+2 pi i k / (4p)}, w^2 and w^3 by complex products
              const cplx<float> w1 = twiddle_f32(k, lp + 2, inverse);
              const cplx<float> w2 = cmul(w1, w1);
              const cplx<float> w3 = cmul(w1, w2);
              a1 = cmul(a1, w1);
              a2 = cmul(a2, w2);
              a3 = cmul(a3, w3);
            } else {
              int e = k << tshift;
              a1 = cmul_tw(a1, tw[e], inverse);
              a2 = cmul_tw(a2, tw[2 * e], inverse);
              a3 = cmul_tw(a3, tw[3 * e], inverse);
            }
          } else {
            int e = k << tshift;
            a1 = cmul_tw(a1, tw[e], inverse);
            a2 = cmul_tw(a2, tw[2 * e], inverse);
            a3 = cmul_tw(a3, tw[3 * e], inverse);
          }
        }
        cplx<T> s02 = a0 + a2, d02 = a0 - a2;
        cplx<T> s13 = a1 + a3, d13 = a1 - a3;
        // 4-point DFT: y1 = d02 + s d13 with s = -i (forward) or +i (inverse)
        cplx<T> r13 = inverse ? mul_pi(d13) : mul_mi(d13);
        y[b][0] = s02 + s13;
        y[b][1] = d02 + r13;
        y[b][2] = s02 - s13;
        y[b][3] = d02 - r13;
        dst[b] = ((i - k) << 2) + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      int i = t + b * NT;
      if (i < q) {
        buf[dst[b]] = y[b][0];
        buf[dst[b] + p] = y[b][1];
        buf[dst[b] + 2 * p] = y[b][2];
        buf[dst[b] + 3 * p] = y[b][3];
      }
    }
    __syncthreads();
    p <<= 2;
    lp += 2;
  }
}

// -------------------------------------------------------------------------------------
// Batched form of cta_fft: nb independent sequences of length n in shared memory, sequence
// s starting at buf + s * stride.  Butterflies of all sequences are spread over the CTA
// (nb n/4 <= MAXB NT).  Same Stockham stages and barriers as cta_fft.
// -------------------------------------------------------------------------------------
template <typename T, int NT, int MAXB>
__device__ __forceinline__ void cta_fft_batch(cplx<T>* buf, int n, int log2n, int nb, int stride,
                                              bool inverse, const cplx<T>* __restrict__ tw) {
  const int t = threadIdx.x;
  int p = 1, lp = 0;
  if (log2n & 1) {
    const int h = n >> 1, tot = nb * h;
    cplx<T> y0[2 * MAXB], y1[2 * MAXB];
    int dst[2 * MAXB];
#pragma unroll
    for (int b = 0; b < 2 * MAXB; ++b) {
      int g = t + b * NT;
      if (g < tot) {
        int s = g >> (log2n - 1), i = g & (h - 1);
        cplx<T>* q = buf + s * stride;
        cplx<T> a0 = q[i], a1 = q[i + h];
        y0[b] = a0 + a1;
        y1[b] = a0 - a1;
        dst[b] = s * stride + i * 2;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 2 * MAXB; ++b) {
      int g = t + b * NT;
      if (g < tot) {
        buf[dst[b]] = y0[b];
        buf[dst[b] + 1] = y1[b];
      }
    }
    __syncthreads();
    p = 2;
    lp = 1;
  }
  const int qn = n >> 2, tot = nb * qn;
  while (p < n) {
    cplx<T> y[MAXB][4];
    int dst[MAXB];
    const int tshift = kTwiddleLog2 - lp - 2;
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      int g = t + b * NT;
      if (g < tot) {
        int s = g >> (log2n - 2), i = g & (qn - 1);
        const cplx<T>* q = buf + s * stride;
        int k = i & (p - 1);
        cplx<T> a0 = q[i], a1 = q[i + qn], a2 = q[i + 2 * qn], a3 = q[i + 3 * qn];
        if (p > 1) {
          int e = k << tshift;
          a1 = cmul_tw(a1, tw[e], inverse);
          a2 = cmul_tw(a2, tw[2 * e], inverse);
          a3 = cmul_tw(a3, tw[3 * e], inverse);
        }
        cplx<T> s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = a1 - a3;
        cplx<T> r13 = inverse ? mul_pi(d13) : mul_mi(d13);
        y[b][0] = s02 + s13;
        y[b][1] = d02 + r13;
        y[b][2] = s02 - s13;
        y[b][3] = d02 - r13;
        dst[b] = s * stride + ((i - k) << 2) + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      int g = t + b * NT;
      if (g < tot) {
        buf[dst[b]] = y[b][0];
        buf[dst[b] + p] = y[b][1];
        buf[dst[b] + 2 * p] = y[b][2];
        buf[dst[b] + 3 * p] = y[b][3];
      }
    }
    __syncthreads();
    p <<= 2;
    lp += 2;
  }
}

// -------------------------------------------------------------------------------------
// Block reduction of a double (deterministic: fixed shuffle tree, then warp 0 over the
// per-warp partials).  scratch must hold NT/32 doubles.  Result broadcast to all threads.
// -------------------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();                                 // scratch may still be read by a previous call
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < NT / 32) ? scratch[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) scratch[NT / 32] = r;
  }
  __syncthreads();
  return scratch[NT / 32];
}

// Block sum of float partials with double-float (~48-bit) accumulation: warp shuffles of
// (hi, lo) pairs, then warp 0 over the per-warp partials.  No float64 instruction runs
// (on this part each costs ~62 float32 ones).  `slot` (NT/32 df entries) must not be in use
// by another reduction still being read; callers alternate two slots.  After the call only
// warp 0 holds the result; `finish(total_hi, total_lo)` runs on thread 0 before the final
// barrier, so it can publish scalars through shared memory to the whole CTA.
template <int NT, typename Finish>
__device__ __forceinline__ void block_sum_df(float v, df* slot, Finish finish) {
  df a(v, 0.0f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df b(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    a = a + b;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) slot[w] = a;
  __syncthreads();
  if (w == 0) {
    df r = (l < NT / 32) ? slot[l] : df(0.0f, 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df b(__shfl_xor_sync(0xffffffffu, r.hi, o), __shfl_xor_sync(0xffffffffu, r.lo, o));
      r = r + b;
    }
    if (l == 0) finish(r.hi, r.lo);
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  if (w == 0) {
    double r = (l < NT / 32) ? scratch[l] : -1.0e308;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (l == 0) scratch[NT / 32] = r;
  }
  __syncthreads();
  return scratch[NT / 32];
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double* scratch) {
  return -block_max<NT>(-v, scratch);
}

// -------------------------------------------------------------------------------------
// Thread-block clusters: a barrier over every thread of the cluster (release/acquire, so
// shared-memory writes before it are visible to the partner CTA after it), the CTA's rank,
// and the partner CTA's copy of a shared-memory object in a cluster of two.
// -------------------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() { return __clusterRelativeBlockRank(); }
template <typename P>
__device__ __forceinline__ P* peer(P* p) {
  return static_cast<P*>(__cluster_map_shared_rank(static_cast<const void*>(p),
                                                   __clusterRelativeBlockRank() ^ 1u));
}

}  // namespace sgn
