// Register-blocked Stockham FFT for one 1d instance per CTA, with a paired spectral layout.
//
// A length-n transform (n = 2^L) runs on NTA = n/E threads that each hold E = 8 (n >= 256)
// or 4 (n <= 128) elements in registers (8 rather than 16: twice the resident warps, and a
// double-float or float64 stage fits the 64 registers per thread of a 1024-thread CTA).
// Thread t's "natural" elements are x[t + e NTA], e < E.  The transform is a sequence of
// Stockham stages: a stage of radix R at sub-transform length P takes butterfly i's inputs
// x[i + r n/R], twiddles them by
// w^{r k} (w = e^{-+2 pi i/(P R)}, k = i mod P), applies the R-point DFT, and writes output
// s to ((i - k) R + k) + s P.  Every stage but the paired one gives each thread E/R
// butterflies whose inputs are its natural elements, so a stage is: compute in registers,
// write the outputs to shared memory, barrier, read the natural elements of the next stage.
// A length-n transform needs 2-4 such exchanges instead of log2(n)/2 radix-4 passes.
//
// Paired stage.  The last forward stage (first inverse stage) has radix RP = E/2 and
// P = 2 NTA; thread t owns butterflies i_0 = t and i_1 = 2 NTA - t (thread 0: i_1 = NTA).
// Its E outputs are the spectral coefficients X[i_b + s 2 NTA], s < RP, held in register
// b RP + s, and the mirror n - m of each of them lies in the same thread.  So everything a
// spectral step needs for mode m and n - m (unpacking two real fields from one complex
// transform, Hermitian symmetry, the G-matvec's mode pairing, dot products) is local to a
// thread, and spectral vectors can stay in registers between iterations.
//
// Shared-memory layout: 8-byte elements (float2 for float32; two planes of float2 for
// double-float, high and low parts; two planes of double for float64, real and imaginary
// parts) addressed through a GF(2)-linear XOR swizzle of the element index.  The swizzle
// matrix was chosen by search so that every access pattern of the stage plans below
// touches 16 distinct 8-byte bank pairs per half-warp, except the reversed half of the
// paired stage (one 2-way conflict per half-warp, which no per-block permutation avoids).
// Linearity lets every address be formed as (per-thread base) XOR (compile-time constant).
#pragma once
#include <type_traits>

#include "sgn_common.cuh"

namespace sgn {
namespace f1 {

template <int V>
using IC = std::integral_constant<int, V>;

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    static_for<B + 1, E>(f);
  }
}

// ---------------------------------------------------------------------------------------
// Stage plan for n = 2^L.
// ---------------------------------------------------------------------------------------
template <int L>
struct Plan {
  static constexpr int n = 1 << L;
  static constexpr int LE = L >= 8 ? 3 : 2;                 // log2 elements per thread
  static constexpr int E = 1 << LE;
  static constexpr int LP = LE - 1;                          // log2 radix of the paired stage
  static constexpr int RP = 1 << LP;
  static constexpr int HS = RP / 2;                          // half-spectrum slots per butterfly
  static constexpr int LNTA = L - LE;
  static constexpr int NTA = n / E;                          // threads holding data
  static constexpr int NT = NTA < 32 ? 32 : NTA;             // threads per CTA
  static constexpr bool kIdle = NT > NTA;
  static constexpr int REST = L - LP;                        // bits of the plain stages
  static constexpr int NS = (REST + LE - 1) / LE;            // number of plain stages
  // log2 radix of plain stage q (as even a split as possible, larger ones first)
  static constexpr int bits(int q) { return REST / NS + (q < REST % NS ? 1 : 0); }
  // log2 P of plain stage q in the forward transform (stages 0..NS-1, then the paired one)
  static constexpr int lp_fwd(int q) {
    int s = 0;
    for (int i = 0; i < q; ++i) s += bits(i);
    return s;
  }
  // log2 P of plain stage q in the inverse transform (paired stage first, then q = NS-1..0)
  static constexpr int lp_inv(int q) {
    int s = LP;
    for (int i = q + 1; i < NS; ++i) s += bits(i);
    return s;
  }
  // CTAs per SM the kernels are compiled for: one CTA of NT >= 512 threads (65536 / NT
  // registers per thread), else enough CTAs for 512 threads (128 registers per thread)
  static constexpr int kMinBlocks = NT >= 512 ? 1 : 512 / NT;
};

// ---------------------------------------------------------------------------------------
// Swizzle: a -> a ^ key(a >> 4), key a 4 x 10 matrix over GF(2) given by its row masks.
// ---------------------------------------------------------------------------------------
constexpr int kSwRow0 = 823, kSwRow1 = 49, kSwRow2 = 261, kSwRow3 = 303;

__host__ __device__ constexpr int parity_c(int v) {
  v ^= v >> 16;
  v ^= v >> 8;
  v ^= v >> 4;
  v ^= v >> 2;
  v ^= v >> 1;
  return v & 1;
}
// compile-time form (constant-folded after unrolling)
__host__ __device__ constexpr int swz_c(int a) {
  const int h = a >> 4;
  return a ^ (parity_c(h & kSwRow0) | (parity_c(h & kSwRow1) << 1) |
              (parity_c(h & kSwRow2) << 2) | (parity_c(h & kSwRow3) << 3));
}
__device__ __forceinline__ int swz(int a) {
  const int h = a >> 4;
  return a ^ ((__popc(h & kSwRow0) & 1) | ((__popc(h & kSwRow1) & 1) << 1) |
              ((__popc(h & kSwRow2) & 1) << 2) | ((__popc(h & kSwRow3) & 1) << 3));
}

// ---------------------------------------------------------------------------------------
// Exchange buffer of n complex elements in 8-byte planes (see the header comment).
// ---------------------------------------------------------------------------------------
template <typename T>
struct XBuf;

template <>
struct XBuf<float> {
  cplx<float>* p;
  __device__ __forceinline__ XBuf(void* base, int) : p(static_cast<cplx<float>*>(base)) {}
  __device__ __forceinline__ void st(int a, cplx<float> v) const { p[a] = v; }
  __device__ __forceinline__ cplx<float> ld(int a) const { return p[a]; }
};

template <>
struct XBuf<df> {
  float2* hi;
  float2* lo;
  __device__ __forceinline__ XBuf(void* base, int n)
      : hi(static_cast<float2*>(base)), lo(static_cast<float2*>(base) + n) {}
  __device__ __forceinline__ void st(int a, cplx<df> v) const {
    hi[a] = make_float2(v.x.hi, v.y.hi);
    lo[a] = make_float2(v.x.lo, v.y.lo);
  }
  __device__ __forceinline__ cplx<df> ld(int a) const {
    const float2 h = hi[a], l = lo[a];
    return mk(df(h.x, l.x), df(h.y, l.y));
  }
};

template <>
struct XBuf<double> {
  double* re;
  double* im;
  __device__ __forceinline__ XBuf(void* base, int n)
      : re(static_cast<double*>(base)), im(static_cast<double*>(base) + n) {}
  __device__ __forceinline__ void st(int a, cplx<double> v) const {
    re[a] = v.x;
    im[a] = v.y;
  }
  __device__ __forceinline__ cplx<double> ld(int a) const { return mk(re[a], im[a]); }
};

// ---------------------------------------------------------------------------------------
// Constants in the working precision and fixed rotations.  Every constant is split into
// its float32 parts in a constexpr context, so no float64 arithmetic reaches the device.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T kc(double d, float hi, float lo);
template <>
__device__ __forceinline__ float kc<float>(double, float hi, float) { return hi; }
template <>
__device__ __forceinline__ double kc<double>(double d, float, float) { return d; }
template <>
__device__ __forceinline__ df kc<df>(double, float hi, float lo) { return df(hi, lo); }

// cos and sin of 2 pi m / 16, m = 0..15
constexpr double kCos16[16] = {1.0,
                               0.92387953251128675613,
                               0.70710678118654752440,
                               0.38268343236508977173,
                               0.0,
                               -0.38268343236508977173,
                               -0.70710678118654752440,
                               -0.92387953251128675613,
                               -1.0,
                               -0.92387953251128675613,
                               -0.70710678118654752440,
                               -0.38268343236508977173,
                               0.0,
                               0.38268343236508977173,
                               0.70710678118654752440,
                               0.92387953251128675613};
constexpr double kSin16(int m) { return kCos16[(m + 12) & 15]; }   // sin x = cos(x - pi/2)

// a * e^{-2 pi i M / 16}.  Multiples of 4 are free, odd multiples of 2 cost two products.
template <typename T, int M>
__device__ __forceinline__ cplx<T> rot16c(cplx<T> a) {
  constexpr int m = M & 15;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return mk(a.y, -a.x);
  } else if constexpr (m == 8) {
    return mk(-a.x, -a.y);
  } else if constexpr (m == 12) {
    return mk(-a.y, a.x);
  } else if constexpr ((m & 1) == 0) {
    constexpr double d = kCos16[2];
    constexpr float hi = (float)d, lo = (float)(d - (double)hi);
    const T r = kc<T>(d, hi, lo);
    if constexpr (m == 2) return mk((a.x + a.y) * r, (a.y - a.x) * r);
    if constexpr (m == 6) return mk((a.y - a.x) * r, -((a.x + a.y) * r));
    if constexpr (m == 10) return mk(-((a.x + a.y) * r), (a.x - a.y) * r);
    if constexpr (m == 14) return mk((a.x - a.y) * r, (a.x + a.y) * r);
  } else {
    // e^{-i theta}: (x c + y s, y c - x s)
    constexpr double c = kCos16[m], s = kSin16(m);
    constexpr float ch = (float)c, cl = (float)(c - (double)ch);
    constexpr float sh = (float)s, sl = (float)(s - (double)sh);
    const T cc = kc<T>(c, ch, cl), ss = kc<T>(s, sh, sl);
    return mk(a.x * cc + a.y * ss, a.y * cc - a.x * ss);
  }
}

// the same with m known only after unrolling
template <typename T>
__device__ __forceinline__ cplx<T> rot16(cplx<T> a, int m) {
  switch (m & 15) {
    case 0: return a;
    case 1: return rot16c<T, 1>(a);
    case 2: return rot16c<T, 2>(a);
    case 3: return rot16c<T, 3>(a);
    case 4: return rot16c<T, 4>(a);
    case 5: return rot16c<T, 5>(a);
    case 6: return rot16c<T, 6>(a);
    case 7: return rot16c<T, 7>(a);
    case 8: return rot16c<T, 8>(a);
    case 9: return rot16c<T, 9>(a);
    case 10: return rot16c<T, 10>(a);
    case 11: return rot16c<T, 11>(a);
    case 12: return rot16c<T, 12>(a);
    case 13: return rot16c<T, 13>(a);
    case 14: return rot16c<T, 14>(a);
    default: return rot16c<T, 15>(a);
  }
}

// In-register DFT of R = 1, 2, 4, 8, 16 points, outputs in natural order.  R = 8 and 16 are
// one Cooley-Tukey split (2 x 4 and 4 x 4) with fixed internal twiddles.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft(cplx<T> (&a)[R]) {
  if constexpr (R == 2) {
    const cplx<T> d = a[0] - a[1];
    a[0] = a[0] + a[1];
    a[1] = d;
  } else if constexpr (R == 4) {
    const cplx<T> s02 = a[0] + a[2], d02 = a[0] - a[2];
    const cplx<T> s13 = a[1] + a[3], d13 = a[1] - a[3];
    const cplx<T> r13 = INV ? mul_pi(d13) : mul_mi(d13);
    a[0] = s02 + s13;
    a[1] = d02 + r13;
    a[2] = s02 - s13;
    a[3] = d02 - r13;
  } else if constexpr (R == 8 || R == 16) {
    constexpr int R1 = (R == 8) ? 2 : 4, R2 = R / R1;
    cplx<T> u[R];                                  // u[n2 R1 + k1]
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      cplx<T> b[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) b[n1] = a[R2 * n1 + n2];
      dft<T, R1, INV>(b);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int m = (n2 * k1 * (16 / R)) & 15;   // W_R^{n2 k1} = W_16^{m}
        u[n2 * R1 + k1] = rot16(b[k1], INV ? 16 - m : m);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cplx<T> c[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) c[n2] = u[n2 * R1 + k1];
      dft<T, R2, INV>(c);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = c[k2];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Stage twiddles: a[r] *= w^r, w = e^{-+2 pi i k / 2^LPR}, r = 1..R-1.
// ---------------------------------------------------------------------------------------
// float32: computed in registers from at most three sincospif values; every w^r is at most
// three complex products away from one of them.
struct TwF32 {
  template <int R, int LPR, bool INV>
  __device__ __forceinline__ void apply(cplx<float> (&a)[R], int k) const {
    if constexpr (R >= 2) {
      const cplx<float> w1 = twiddle_f32(k, LPR, INV);
      a[1] = cmul(a[1], w1);
      if constexpr (R >= 4) {
        const cplx<float> w2 = cmul(w1, w1), w3 = cmul(w1, w2);
        a[2] = cmul(a[2], w2);
        a[3] = cmul(a[3], w3);
        if constexpr (R >= 8) {
          const cplx<float> w4 = twiddle_f32(4 * k, LPR, INV);
          a[4] = cmul(a[4], w4);
          a[5] = cmul(a[5], cmul(w4, w1));
          a[6] = cmul(a[6], cmul(w4, w2));
          a[7] = cmul(a[7], cmul(w4, w3));
          if constexpr (R == 16) {
            const cplx<float> w8 = twiddle_f32(8 * k, LPR, INV), w12 = cmul(w4, w8);
            a[8] = cmul(a[8], w8);
            a[9] = cmul(a[9], cmul(w8, w1));
            a[10] = cmul(a[10], cmul(w8, w2));
            a[11] = cmul(a[11], cmul(w8, w3));
            a[12] = cmul(a[12], w12);
            a[13] = cmul(a[13], cmul(w12, w1));
            a[14] = cmul(a[14], cmul(w12, w2));
            a[15] = cmul(a[15], cmul(w12, w3));
          }
        }
      }
    }
  }
};

// double-float and float64: table of e^{-2 pi i j / 2^kTwiddleLog2}
template <typename T>
struct TwTab {
  const cplx<T>* __restrict__ tw;
  template <int R, int LPR, bool INV>
  __device__ __forceinline__ void apply(cplx<T> (&a)[R], int k) const {
#pragma unroll
    for (int r = 1; r < R; ++r) a[r] = cmul_tw(a[r], tw[(r * k) << (kTwiddleLog2 - LPR)], INV);
  }
};

template <typename T>
struct TwOf {
  using type = TwTab<T>;
};
template <>
struct TwOf<float> {
  using type = TwF32;
};

// ---------------------------------------------------------------------------------------
// Stages.
// ---------------------------------------------------------------------------------------
template <typename T, int L, int LR, int LPW, bool INV, typename Tw>
__device__ __forceinline__ void stage_compute(cplx<T> (&v)[Plan<L>::E], int t, const Tw& tw) {
  using PL = Plan<L>;
  constexpr int R = 1 << LR, BB = PL::E / R;
#pragma unroll
  for (int j = 0; j < BB; ++j) {
    cplx<T> a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = v[j + r * BB];
    if constexpr (LPW > 0) {
      const int k = (t + j * PL::NTA) & ((1 << LPW) - 1);
      tw.template apply<R, LPW + LR, INV>(a, k);
    }
    dft<T, R, INV>(a);
#pragma unroll
    for (int s = 0; s < R; ++s) v[j + s * BB] = a[s];
  }
}

// Stockham address of output s of butterfly i: (i mod P) | s << LPW | (i div P) << (LPW+LR)
template <int LR, int LPW>
__host__ __device__ constexpr int stock_addr(int i, int s) {
  return (i & ((1 << LPW) - 1)) | (s << LPW) | ((i >> LPW) << (LPW + LR));
}

template <typename T, int L, int LR, int LPW>
__device__ __forceinline__ void stage_write(const XBuf<T>& X, const cplx<T> (&v)[Plan<L>::E],
                                            int t) {
  using PL = Plan<L>;
  constexpr int R = 1 << LR, BB = PL::E / R;
  const int base = swz(stock_addr<LR, LPW>(t, 0));
#pragma unroll
  for (int j = 0; j < BB; ++j)
#pragma unroll
    for (int s = 0; s < R; ++s)
      X.st(base ^ swz_c(stock_addr<LR, LPW>(j * PL::NTA, s)), v[j + s * BB]);
}

template <typename T, int L>
__device__ __forceinline__ void read_natural(const XBuf<T>& X, cplx<T> (&v)[Plan<L>::E],
                                             int bnat) {
  using PL = Plan<L>;
#pragma unroll
  for (int e = 0; e < PL::E; ++e) v[e] = X.ld(bnat ^ swz_c(e * PL::NTA));
}

// Per-thread geometry of the layouts.  `odd` selects the pairing of the odd-mode half of a
// two-CTA transform (see the cluster section below): butterflies t and 2 NTA - 1 - t, whose
// outputs k and N - 1 - k (N = 2^L) are the local indices of the global mirror pair there.
template <int L>
struct Geo {
  using PL = Plan<L>;
  int t;
  bool act;            // holds data (t < NTA)
  int i1;              // second paired butterfly
  int bnat;            // swz(t)
  int bp0, bp1;        // swz(i_0), swz(i_1): paired reads
  int bw0, bw1;        // swz(i_0 RP), swz(i_1 RP): paired writes
  __device__ __forceinline__ explicit Geo(int tt, bool odd = false) : t(tt) {
    act = !PL::kIdle || t < PL::NTA;
    i1 = odd ? 2 * PL::NTA - 1 - t : ((t == 0) ? PL::NTA : 2 * PL::NTA - t);
    bnat = swz(t);
    bp0 = bnat;
    bp1 = swz(i1);
    bw0 = swz(t << PL::LP);
    bw1 = swz(i1 << PL::LP);
  }
  // spectral index of register b RP + s in the paired layout
  __device__ __forceinline__ int mode(int b, int s) const {
    return (b ? i1 : t) + s * 2 * PL::NTA;
  }
};

// Forward transform: natural registers in, paired registers out.  All NT threads call.
// Starts with a barrier (earlier readers of X are done) and leaves X free for reuse only
// after the caller's next barrier.
template <typename T, int L, typename Tw>
__device__ __forceinline__ void fft_fwd(const XBuf<T>& X, cplx<T> (&v)[Plan<L>::E],
                                        const Geo<L>& g, const Tw& tw) {
  using PL = Plan<L>;
  static_for<0, PL::NS>([&](auto Q) {
    constexpr int q = decltype(Q)::value;
    constexpr int LR = PL::bits(q), LPW = PL::lp_fwd(q);
    if (g.act) stage_compute<T, L, LR, LPW, false>(v, g.t, tw);
    __syncthreads();
    if (g.act) stage_write<T, L, LR, LPW>(X, v, g.t);
    __syncthreads();
    if (g.act) {
      if constexpr (q + 1 < PL::NS) {
        read_natural<T, L>(X, v, g.bnat);
      } else {
#pragma unroll
        for (int r = 0; r < PL::RP; ++r) {
          const int c = swz_c(r * 2 * PL::NTA);
          v[r] = X.ld(g.bp0 ^ c);
          v[PL::RP + r] = X.ld(g.bp1 ^ c);
        }
      }
    }
  });
  if (g.act) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      cplx<T> a[PL::RP];
#pragma unroll
      for (int r = 0; r < PL::RP; ++r) a[r] = v[b * PL::RP + r];
      tw.template apply<PL::RP, L, false>(a, b ? g.i1 : g.t);
      dft<T, PL::RP, false>(a);
#pragma unroll
      for (int s = 0; s < PL::RP; ++s) v[b * PL::RP + s] = a[s];
    }
  }
}

// Inverse transform (unnormalised): paired registers in, natural registers out.
template <typename T, int L, typename Tw>
__device__ __forceinline__ void fft_inv(const XBuf<T>& X, cplx<T> (&v)[Plan<L>::E],
                                        const Geo<L>& g, const Tw& tw) {
  using PL = Plan<L>;
  if (g.act) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      cplx<T> a[PL::RP];
#pragma unroll
      for (int r = 0; r < PL::RP; ++r) a[r] = v[b * PL::RP + r];
      dft<T, PL::RP, true>(a);
#pragma unroll
      for (int s = 0; s < PL::RP; ++s) v[b * PL::RP + s] = a[s];
    }
  }
  __syncthreads();
  if (g.act) {
#pragma unroll
    for (int s = 0; s < PL::RP; ++s) {
      X.st(g.bw0 ^ s, v[s]);
      X.st(g.bw1 ^ s, v[PL::RP + s]);
    }
  }
  __syncthreads();
  if (g.act) read_natural<T, L>(X, v, g.bnat);
  static_for<0, PL::NS>([&](auto Q) {
    constexpr int q = PL::NS - 1 - decltype(Q)::value;
    constexpr int LR = PL::bits(q), LPW = PL::lp_inv(q);
    if (g.act) stage_compute<T, L, LR, LPW, true>(v, g.t, tw);
    if constexpr (q > 0) {
      __syncthreads();
      if (g.act) stage_write<T, L, LR, LPW>(X, v, g.t);
      __syncthreads();
      if (g.act) read_natural<T, L>(X, v, g.bnat);
    }
  });
}

// ---------------------------------------------------------------------------------------
// Half-spectrum slots of the paired layout.  Slot (b, s), s < HS, is mode i_b + s 2 NTA
// (all below n/2); thread 0 also owns the Nyquist mode n/2 in register HS.  The mirror
// n - m of a slot sits in register mirror(b, s).  `t0` selects thread 0's pairing; the
// odd half of a two-CTA transform passes false on every thread (its pairing has no
// self-paired butterfly).
// ---------------------------------------------------------------------------------------
template <int L, typename V>
__device__ __forceinline__ V mirror_get(const V (&v)[Plan<L>::E], bool t0, int b, int s) {
  using PL = Plan<L>;
  // b and s are compile-time after unrolling: a select between two fixed registers
  if (b == 0) {
    const V x = v[(PL::RP - s) & (PL::RP - 1)], y = v[2 * PL::RP - 1 - s];
    return t0 ? x : y;
  }
  const V x = v[2 * PL::RP - 1 - s], y = v[PL::RP - 1 - s];
  return t0 ? x : y;
}
template <int L, typename V>
__device__ __forceinline__ void mirror_set(V (&v)[Plan<L>::E], bool t0, int b, int s, V val) {
  using PL = Plan<L>;
  if (b == 0) {
    if (t0) v[(PL::RP - s) & (PL::RP - 1)] = val;
    else v[2 * PL::RP - 1 - s] = val;
  } else {
    if (t0) v[2 * PL::RP - 1 - s] = val;
    else v[PL::RP - 1 - s] = val;
  }
}

// ---------------------------------------------------------------------------------------
// Compact in-shared-memory transform for the double-float and float64 paths.
//
// The register-resident transforms above are fully unrolled, which for double-float and
// float64 arithmetic makes hundreds of kilobytes of code per call site and stalls on
// instruction fetch.  fft_smem runs the same Stockham stages with the data in the exchange
// buffer between stages, natural order in and out: a stage reads the thread's natural
// elements, waits at a barrier, computes its butterflies and writes their outputs in
// Stockham order, and waits again.  Stages of equal radix share one code body through a
// runtime stage loop, only the forward transform exists (callers form the inverse as
// conj(F(conj x))), and the function is not inlined, so every caller runs the same code.
// ---------------------------------------------------------------------------------------
template <int L>
struct SmemPlan {
  static constexpr int LE = Plan<L>::LE;
  static constexpr int NS = (L + LE - 1) / LE;
  static constexpr int bits(int q) { return L / NS + (q < L % NS ? 1 : 0); }
  static constexpr bool uses(int lr) {
    for (int q = 0; q < NS; ++q)
      if (bits(q) == lr) return true;
    return false;
  }
};

template <typename T, int L, int LR>
__device__ __forceinline__ void smem_stage(const XBuf<T>& X, int t, int bnat, int lp,
                                           const cplx<T>* __restrict__ tw) {
  using PL = Plan<L>;
  constexpr int E = PL::E, NTA = PL::NTA, R = 1 << LR, BB = E / R;
  const bool act = !PL::kIdle || t < NTA;
  cplx<T> v[E];
  if (act) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = X.ld(bnat ^ swz_c(e * NTA));
  }
  __syncthreads();
  if (act) {
    const int pm = (1 << lp) - 1, sh = kTwiddleLog2 - lp - LR;
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      const int i = t + j * NTA, k = i & pm;
      const int base = k | ((i >> lp) << (lp + LR));
      cplx<T> a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = v[j + r * BB];
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) a[r] = cmul(a[r], tw[(r * k) << sh]);
      }
      dft<T, R, false>(a);
#pragma unroll
      for (int s = 0; s < R; ++s) X.st(swz(base | (s << lp)), a[s]);
    }
  }
  __syncthreads();
}

// Forward transform of the n = 2^L elements in X (natural order in and out).  All threads
// of the CTA call; entered and left at a barrier-consistent point (the caller's writes of
// the input must be complete, or be the caller's own natural elements).
template <typename T, int L>
__device__ __noinline__ void fft_smem(const XBuf<T> X, const cplx<T>* __restrict__ tw) {
  using SP = SmemPlan<L>;
  const int t = threadIdx.x;
  const int bnat = swz(t);
  int lp = 0;
#pragma unroll 1
  for (int q = 0; q < SP::NS; ++q) {
    const int lr = SP::bits(q);
    if constexpr (SP::uses(4)) if (lr == 4) smem_stage<T, L, 4>(X, t, bnat, lp, tw);
    if constexpr (SP::uses(3)) if (lr == 3) smem_stage<T, L, 3>(X, t, bnat, lp, tw);
    if constexpr (SP::uses(2)) if (lr == 2) smem_stage<T, L, 2>(X, t, bnat, lp, tw);
    if constexpr (SP::uses(1)) if (lr == 1) smem_stage<T, L, 1>(X, t, bnat, lp, tw);
    lp += lr;
  }
}

// ---------------------------------------------------------------------------------------
// Two-CTA transforms: an instance of n = 2 N points (N = 2^L) on a thread-block cluster of
// two CTAs.  Rank r holds the real-space points [r N, r N + N) and the spectral modes
// m = 2 k + r (k < N) at local index k: one radix-2 stage across the pair plus a local
// length-N transform on each CTA.
//   forward (decimation in frequency): y_r[j] = (x[j] + (-1)^r x[j + N]) w^{r j}, then
//     Y_r = F_N(y_r), so Y_r[k] = X[2 k + r] (w = e^{-2 pi i / n});
//   after a forward transform that computes an inverse as conj(F(conj X)):
//     u_r = F_N(conj X_r), conj(x)[j] = u_0[j] + w^j u_1[j], conj(x)[j + N] = u_0 - w^j u_1;
//   after a true inverse transform: z_r = F_N^{-1}(X_r), x[j] = z_0 + w^{-j} z_1,
//     x[j + N] = z_0 - w^{-j} z_1.
// The global mirror n - m of mode m = 2 k + r has local index N - k (mod N) on rank 0 (the
// ordinary paired layout) and N - 1 - k on rank 1 (Geo's odd pairing).  The exchange runs
// through distributed shared memory: each CTA publishes its natural elements in its own
// exchange buffer, the pair meets at a cluster barrier, each reads the partner's elements
// at the same positions, and a second barrier ends the reads before either buffer is
// written again.
// ---------------------------------------------------------------------------------------
// e^{-+2 pi i j / 2^LG} in number type T (float32 from sincospif, else from the table)
template <typename T, int LG>
__device__ __forceinline__ cplx<T> xtw(int j, bool inv, const cplx<T>* __restrict__ tw) {
  if constexpr (std::is_same<T, float>::value) {
    return twiddle_f32(j, LG, inv);
  } else {
    const cplx<T> w = tw[j << (kTwiddleLog2 - LG)];
    return inv ? conj(w) : w;
  }
}

enum CrossKind { kSplitFwd = 0, kJoinConj = 1, kJoinInv = 2 };

// The cross-CTA stage on the thread's natural elements v[e] (local j = t + e NTA), through
// the exchange buffers X (own) and XP (partner).  All threads of both CTAs call it.
template <typename T, int L, int KIND>
__device__ __forceinline__ void cross(const XBuf<T>& X, const XBuf<T>& XP,
                                      cplx<T> (&v)[Plan<L>::E], int t, int bnat, bool act,
                                      unsigned r, const cplx<T>* __restrict__ tw) {
  using PL = Plan<L>;
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) {
      cplx<T> a = v[e];
      if (KIND != kSplitFwd && r)
        a = cmul(a, xtw<T, L + 1>(t + e * PL::NTA, KIND == kJoinInv, tw));
      v[e] = a;
      X.st(bnat ^ swz_c(e * PL::NTA), a);
    }
  }
  cluster_sync();
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) {
      const cplx<T> b = XP.ld(bnat ^ swz_c(e * PL::NTA));
      if (!r) {
        v[e] = v[e] + b;
      } else if (KIND == kSplitFwd) {
        v[e] = cmul(b - v[e], xtw<T, L + 1>(t + e * PL::NTA, false, tw));
      } else {
        v[e] = b - v[e];
      }
    }
  }
  cluster_sync();
}

// The same on the natural elements held in X (the state around fft_smem).
template <typename T, int L, int KIND>
__device__ __forceinline__ void cross_smem(const XBuf<T>& X, const XBuf<T>& XP, int t,
                                           int bnat, bool act, unsigned r,
                                           const cplx<T>* __restrict__ tw) {
  using PL = Plan<L>;
  cplx<T> v[PL::E];
  if (act) read_natural<T, L>(X, v, bnat);
  cross<T, L, KIND>(X, XP, v, t, bnat, act, r, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < PL::E; ++e) X.st(bnat ^ swz_c(e * PL::NTA), v[e]);
  }
}

}  // namespace f1
}  // namespace sgn
