// Mixed-radix Stockham FFT in shared (or global) memory for lengths n = 2^a 3^b 5^c
// (a >= 1): radix-8 stages, one radix-4 or radix-2 stage, then radix-5 and radix-3 stages,
// two buffers used in turn, and a twiddle table of n - 1 entries per length (the block of
// the stage at sub-length p starts at p - 1 and holds w^{r k}, w = e^{-2 pi i / (p R)},
// r = 1..R-1, k = 0..p-1).  Used by the 1d generic kernels and the 2d row and column passes.
#pragma once
#include "sgn_common.cuh"

namespace sgn {
namespace mr {

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

// One radix-R Stockham stage at sub-length p over nb sequences of length n stored back to
// back: butterfly i of a sequence reads src[i + r n/R], twiddles by w^{r k} (k = i mod p,
// table block at p - 1: entry (r - 1) p + k), writes output s to dst[(i - k) R + k + s p].
// NT threads share the butterflies of all sequences.
template <typename T, int R, int NT>
__device__ __forceinline__ void mr_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                         int n, int p, bool inv, const cplx<T>* __restrict__ tw,
                                         int nb) {
  const int q = n / R;
  auto butterfly = [&](const cplx<T>* __restrict__ sr, cplx<T>* __restrict__ ds, int i, int k) {
    cplx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = sr[i + r * q];
    if (p > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul_tw(x[r], tw[p - 1 + (r - 1) * p + k], inv);
    }
    mr_dft<T, R>(x, inv);
    const int o = (i - k) * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) ds[o + s * p] = x[s];
  };
  if (nb == 1) {
    // one sequence: butterfly i = t, and k = i mod p carried from one butterfly of this
    // thread to its next (i grows by NT) instead of a division each time
    const int step = NT % p;
    int k = threadIdx.x % p;
    for (int i = threadIdx.x; i < q; i += NT) {
      butterfly(src, dst, i, k);
      k += step;
      if (k >= p) k -= p;
    }
  } else {
    for (int t = threadIdx.x; t < q * nb; t += NT) {
      const int sq = t / q, i = t - sq * q;
      butterfly(src + (size_t)sq * n, dst + (size_t)sq * n, i, i % p);
    }
  }
  __syncthreads();
}

// The transform of the nb sequences in a (length n each, natural order, back to back) with
// b as the other buffer; returns the buffer holding the result.  Forward: X_m = sum_j x_j
// e^{-2 pi i j m / n}; inverse without the 1/n.  Callers synchronise before it; it returns
// after a barrier.
template <typename T, int NT>
__device__ cplx<T>* mr_fft(cplx<T>* a, cplx<T>* b, const MrPlan& P, bool inv,
                           const cplx<T>* tw, int nb = 1) {
  cplx<T>* src = a;
  cplx<T>* dst = b;
  int p = 1;
  for (int st = 0; st < P.ns; ++st) {
    const int R = P.radix(st);
    if (R == 8) mr_stage<T, 8, NT>(src, dst, P.n, p, inv, tw, nb);
    else if (R == 4) mr_stage<T, 4, NT>(src, dst, P.n, p, inv, tw, nb);
    else if (R == 2) mr_stage<T, 2, NT>(src, dst, P.n, p, inv, tw, nb);
    else if (R == 5) mr_stage<T, 5, NT>(src, dst, P.n, p, inv, tw, nb);
    else mr_stage<T, 3, NT>(src, dst, P.n, p, inv, tw, nb);
    p *= R;
    cplx<T>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

namespace {

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

}  // namespace

}  // namespace mr
}  // namespace sgn
