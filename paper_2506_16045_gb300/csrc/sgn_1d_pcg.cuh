// a5/a6: preconditioned conjugate gradients for G_{eta,h} x = b in 1d (§3.2, Eq:PCGLinSyst,
// preconditioner A of §4), one CTA per instance, in spectral space (see sgn_1d.cu for the
// formulation) on the register-blocked FFT of sgn_fft1d.cuh.
//
//   MIXED = false: float64 PCG from the caller's initial guess; the Krylov vectors are
//                  half spectra in the workspace, each thread touching only the modes of
//                  its slots (so no barrier guards them).
//   MIXED = true : iterative refinement in double-float (~48-bit) precision.  Each pass
//                  computes the residual r = b - G x with double-float FFTs and
//                  coefficients, stops when sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b), and
//                  otherwise solves G d = r / ||r||_{A^{-1}} by float32 PCG (to rtol_inner,
//                  or adaptively to 0.3 rtol / current ratio within [1e-6, 0.1]) and updates
//                  x += ||r||_{A^{-1}} d in double-float.  The float32 PCG keeps r and p in
//                  registers (the paired spectral layout makes every per-mode step local to
//                  a thread) and the correction d in shared memory; its dot products reduce
//                  in double-float and one thread forms alpha, beta and the stopping test.
//
// n = 16384 runs on a thread-block cluster of two CTAs (CL = 2, sgn_fft1d.cuh's two-CTA
// transforms): each CTA holds half of the points and, in spectral space, the modes of one
// parity; dot products add the two CTAs' block sums in rank order through distributed
// shared memory, so both CTAs take every decision from the same numbers.
//
// Workspace slots per instance (half spectra of n/2 + 1 modes, 16 bytes per mode each):
//   0: b^ (high precision), 1: x^ (high), 2: r^ and 3: p^ (float64 path only).
// The mixed path keeps its double-float coefficients c1, c2, c3 in coef_df (high parts,
// then low parts: 6 floats per point) and float32 copies of eta and h_x in shared memory.
#pragma once
#include <type_traits>

#include "sgn_1d_dev.cuh"
#include "sgn_fft1d.cuh"

namespace sgn {

// Arguments of one solve launch (kernel parameter space: read on use, not held in registers).
struct PcgArgs {
  const Inst1d* insts;
  const int* ids;
  const cplx<double>* tw64;
  const cplx<df>* twdf;
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
  float* coef_df;
  int precision;
  void* ux;             // nullable: also store x_x here (see pcg_body)
};

// LG = log2 n; CL = CTAs per instance (2: thread-block clusters of two CTAs of the
// 2^(LG-1)-point kernel; the only form for LG = 14)
template <int LG, int CL>
cudaError_t pcg1d_launch(const PcgArgs& a, int first, int num, cudaStream_t s);

namespace pcg1d {

using namespace d1;
using f1::Geo;
using f1::Plan;
using f1::XBuf;

// Shared memory of one solve CTA (bytes):
//   [0, 16 n)       exchange planes of the double-float / float64 transforms; the float32
//                   inner solve uses [0, 8 n) for its exchanges and, after them, keeps its
//                   thread-private slot arrays d (correction) and r (residual), [RP + 1][NT]
//                   each, which live only while the inner solve runs;
//   [off_e, +8 n)   (mixed) float32 eta and h_x, from which the inner solve forms its
//                   coefficients.
template <int L>
struct SmemPcg {
  using PL = Plan<L>;
  static constexpr size_t n = (size_t)PL::n;
  static constexpr size_t slot_c = (size_t)(PL::RP + 1) * PL::NT * 8;   // complex float
  static constexpr size_t off_d = 8 * n;
  static constexpr size_t off_r = off_d + slot_c;
  static constexpr size_t end_r = off_r + slot_c;
  static constexpr size_t off_e = ((16 * n > end_r ? 16 * n : end_r) + 15) / 16 * 16;
  static constexpr size_t mixed = off_e + 8 * n;
  static constexpr size_t fp64 = 16 * n;
  static_assert(mixed + 1024 <= 232448, "solve CTA exceeds the shared memory of one SM");
};

// Double-float coefficients of Def:MatrixM in 1d (c1 = eta (1 + h_x^2), c2 = eta^2 h_x / 2,
// c3 = eta^3 / 3) to global memory (high parts, then low parts), and float32 eta, h_x to
// shared memory.  Formed in double-float arithmetic: no float64 instruction.
template <int NT>
__device__ __forceinline__ void prep_coefficients(const double* __restrict__ eta,
                                                  const double* __restrict__ hx, int n,
                                                  float* __restrict__ eh,
                                                  float* __restrict__ cdf) {
  const df third = f1::kc<df>(1.0 / 3.0, (float)(1.0 / 3.0),
                              (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0)));
  for (int j = threadIdx.x; j < n; j += NT) {
    const df e(eta[j]), g(hx[j]);
    const df e2 = e * e;
    const df c[3] = {e + e * g * g, half(e2 * g), e2 * e * third};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cdf[q * n + j] = c[q].hi;
      cdf[(3 + q) * n + j] = c[q].lo;
    }
    eh[j] = e.hi;
    eh[n + j] = g.hi;
  }
}

struct PcgScalars {     // inner float32 PCG
  float rz, alpha, beta;
  int state;            // 0 iterate, 1 converged, 2 breakdown, 3 iteration cap
};

struct PassScalars {    // refinement pass
  double ratio;         // sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b)
  df unscale;           // ||r||_{A^{-1}}
  float scale;          // 1 / ||r||_{A^{-1}}
  float tin2;           // (inner tolerance)^2
  int go;               // 1: run another inner solve
  int status;
};

// Sums over the CTAs of a cluster of CL (1 or 2).  The block's total is published in the
// CTA's slot xs[par]; after a cluster barrier both CTAs add rank 0's and rank 1's totals in
// that order.  Callers flip par after every call, so a slot is rewritten only after the
// partner has passed the next barrier (and so has read it).
template <int NT, int CL, typename Finish>
__device__ __forceinline__ void sum_df(float v, df* slot, df* xs, int& par, Finish finish) {
  if constexpr (CL == 1) {
    block_sum_df<NT>(v, slot, finish);
  } else {
    df* mine = xs + par;
    block_sum_df<NT>(v, slot, [&](float hi, float lo) { *mine = df(hi, lo); });
    cluster_sync();
    if (threadIdx.x == 0) {
      const df o = *peer(mine);
      const df s = cluster_rank() == 0 ? *mine + o : o + *mine;
      finish(s.hi, s.lo);
    }
    __syncthreads();
    par ^= 1;
  }
}

template <int NT, int CL>
__device__ __forceinline__ double sum64(double v, double* red, double* xs, int& par) {
  const double s = block_sum<NT>(v, red);
  if constexpr (CL == 1) {
    return s;
  } else {
    double* mine = xs + par;
    if (threadIdx.x == 0) *mine = s;
    cluster_sync();
    const double o = *peer(mine);
    par ^= 1;
    return cluster_rank() == 0 ? s + o : o + s;
  }
}

// Slot (b, s) of the paired layout for slot number q < RP (compile-time after unrolling).
template <int L>
struct Slot {
  static constexpr int b(int q) { return q / Plan<L>::HS; }
  static constexpr int s(int q) { return q % Plan<L>::HS; }
  static constexpr int reg(int q) { return b(q) * Plan<L>::RP + s(q); }
};

// The solve of one instance by one CTA (CL = 1) or one cluster of two (CL = 2: n = 2^(L+1),
// the CTA of rank r holding points [r nl, r nl + nl) and modes 2 k + r).  With ux non-null
// it also stores x_x (double-float for the mixed path, float64 otherwise) at ux[off + j]:
// the mixed path takes it from the inverse transform of its last refinement pass, which
// yields x + i x_x; the float64 path from its final transform.  A right-hand side that
// follows the solve in a time step then needs one derivative pair less.
template <int L, bool MIXED, int CL>
__device__ __forceinline__ void pcg_body(const PcgArgs& A, int first, void* ux) {
  using PL = Plan<L>;
  using SL = Slot<L>;
  using SM = SmemPcg<L>;
  constexpr int nl = PL::n, E = PL::E, RP = PL::RP, HS = PL::HS, NTA = PL::NTA;
  constexpr int n = CL * nl, h = n / 2;
  constexpr int NT = PL::NT, W = NT / 32;
  using TH = typename std::conditional<MIXED, df, double>::type;   // high precision
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[W + 1];
  __shared__ df slots[2 * W];
  __shared__ PcgScalars sc;
  __shared__ PassScalars ps;
  __shared__ df xs_df[2];
  __shared__ double xs64[2];
  int par = 0;

  const int t = threadIdx.x;
  const unsigned rk = CL > 1 ? cluster_rank() : 0u;
  const Geo<L> g(t, rk != 0);
  const bool t0 = (t == 0);
  const bool ts = t0 && rk == 0;       // owner of the real modes 0 and n/2
  const int id = A.ids[first + (CL > 1 ? (int)(blockIdx.x / CL) : (int)blockIdx.x)];
  const Inst1d I = A.insts[id];
  const long long own = I.off + (long long)rk * nl;    // first point of this CTA
  const double* eta = A.eta + own;
  const double* hx = A.hx + own;
  const double* b = A.b + own;
  double* x = A.x + own;
  const long long S = h + 1;
  // global mode of local spectral index k, and the local index of its mirror n - m
  auto gm = [&](int k) { return CL * k + (int)rk; };
  auto mir = [&](int k) { return rk ? nl - 1 - k : (nl - k) & (nl - 1); };
  auto sum_f = [&](float v, df* sl, auto finish) { sum_df<NT, CL>(v, sl, xs_df, par, finish); };
  auto sum_d = [&](double v) { return sum64<NT, CL>(v, red, xs64, par); };
  cplx<TH>* Bh = reinterpret_cast<cplx<TH>*>(A.ws + I.ws);
  cplx<TH>* Xh = reinterpret_cast<cplx<TH>*>(A.ws + I.ws + S);
  const double rtol = A.rtol, rtol_inner = A.rtol_inner;
  const int maxit = A.maxit, max_refine = A.max_refine;

  // ---- a1: coefficients (or the caller's)
  SolveRec R = {};
  if (A.given) {
    R = A.given[id];
    R.status = SGN_OK;
  } else {
    coeffs_block<NT, CL>(eta, hx, nl, A.kind, red, R);
  }
  R.iters = 0;
  R.refinements = 0;
  R.ratio = 0.0;
  if (R.status != SGN_OK) {
    if (ts) A.rec[id] = R;
    return;
  }
  const double kunit = 2.0 * kPi / I.L;
  const float kf = (float)kunit, sigf = (float)R.sigma, alf = (float)R.alpha;
  const XBuf<TH> XH(smem, nl);
  const XBuf<TH> XHp = CL > 1 ? XBuf<TH>(peer(smem), nl) : XH;   // the partner's
  // float32 preconditioner symbol 1 / (sigma + alpha k^2) of mode m < n/2 (Nyquist: 1/sigma)
  auto dinv = [&](int m) {
    const float k = kf * (float)m;
    return recip(sigf + alf * k * k);
  };
  const float dN = recip(sigf);

  const float* eh = reinterpret_cast<const float*>(smem + SM::off_e);
  const float* cdf = A.coef_df + 6 * own;     // this CTA's points, planes of nl
  if constexpr (MIXED)
    prep_coefficients<NT>(eta, hx, nl, reinterpret_cast<float*>(smem + SM::off_e),
                          A.coef_df + 6 * own);
  const cplx<TH>* twh = MIXED ? reinterpret_cast<const cplx<TH>*>(A.twdf)
                              : reinterpret_cast<const cplx<TH>*>(A.tw64);
  // the cross-CTA stages of CL = 2 around the compact transforms
  auto split_h = [&]() {
    if constexpr (CL > 1) f1::cross_smem<TH, L, f1::kSplitFwd>(XH, XHp, t, g.bnat, g.act, rk, twh);
  };
  auto join_h = [&]() {
    if constexpr (CL > 1) f1::cross_smem<TH, L, f1::kJoinConj>(XH, XHp, t, g.bnat, g.act, rk, twh);
  };

  // ---- b^ and x0^ from one transform of b + i x0
  {
    if (g.act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = t + e * NTA;
        XH.st(g.bnat ^ f1::swz_c(e * NTA), mk(num<TH>(b[j]), num<TH>(x[j])));
      }
    }
    split_h();
    f1::fft_smem<TH, L>(XH, twh);
    float bb = 0.0f;
    if (g.act) {
#pragma unroll
      for (int q = 0; q < RP; ++q) {
        const int k = g.mode(SL::b(q), SL::s(q)), m = gm(k);
        const cplx<TH> y = XH.ld(f1::swz(k));
        const cplx<TH> ym = conj(XH.ld(f1::swz(mir(k))));
        const cplx<TH> s = y + ym, d = mul_mi(y - ym);
        const cplx<TH> bh = mk(half(s.x), half(s.y));
        Bh[m] = bh;
        Xh[m] = mk(half(d.x), half(d.y));
        const float bx = lead(bh.x), by = lead(bh.y);
        bb += ((ts && q == 0) ? 1.0f : 2.0f) * (bx * bx + by * by) * dinv(m);
      }
      if (ts) {
        const cplx<TH> y = XH.ld(f1::swz(nl / 2));
        Bh[h] = mk(y.x, from_int<TH>(0));
        Xh[h] = mk(y.y, from_int<TH>(0));
        const float bx = lead(y.x);
        bb += bx * bx * dN;
      }
    }
    sum_f(bb, slots, [&](float hi, float lo) {
      ps.ratio = (double)hi + (double)lo;        // b.A^{-1}b
    });
  }
  const double bb = ps.ratio;
  const double bnorm = sqrt(bb);
  __syncthreads();                               // ps is reused below
  if (!(bnorm > 0.0)) {
    if (g.act)
#pragma unroll
      for (int e = 0; e < E; ++e) x[t + e * NTA] = 0.0;
    R.status = (bb == 0.0) ? SGN_OK : SGN_ERR_BREAKDOWN;
    if (ts) A.rec[id] = R;
    return;
  }

  int iters = 0;
  int status = SGN_OK;
  if constexpr (!MIXED) {
    // ------------------------------------------------------------------ float64 PCG
    cplx<double>* Rh = A.ws + I.ws + 2 * S;
    cplx<double>* Ph = A.ws + I.ws + 3 * S;
    const CoefGlobal64 coef64{eta, hx};
    const double tol_abs = rtol * bnorm;
    const double inv_n = 1.0 / (double)n;
    const double isig = 1.0 / R.sigma;
    auto dinv64 = [&](int m) {
      const double k = kunit * (double)m;
      return 1.0 / (R.sigma + R.alpha * k * k);
    };
    // conj(Z) of the half spectrum Vh into XH, Z_m = (1 - k) v_m and Z_{n-m} = (1 + k)
    // conj(v_m) (k = 0: the plain inverse), then the transform: XH holds conj(n (v + i v_x))
    auto to_real = [&](const cplx<double>* __restrict__ Vh, bool with_k) {
      __syncthreads();                           // earlier readers of the buffer are done
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int k = g.mode(SL::b(q), SL::s(q)), m = gm(k);
          const double kk = with_k ? kunit * (double)m : 0.0;
          const cplx<double> p = Vh[m];
          if (ts && q == 0) {
            XH.st(0, mk(p.x, 0.0));
          } else {
            XH.st(f1::swz(k), conj(p) * (1.0 - kk));
            XH.st(f1::swz(mir(k)), p * (1.0 + kk));
          }
        }
        if (ts) XH.st(f1::swz(nl / 2), mk(Vh[h].x, 0.0));
      }
      __syncthreads();
      f1::fft_smem<double, L>(XH, A.tw64);
      join_h();
    };
    // (G v)^ of the slots of the half spectrum Vh into gq / gN
    auto matvec = [&](const cplx<double>* __restrict__ Vh, cplx<double>(&gq)[RP],
                      cplx<double>& gN) {
      to_real(Vh, true);
      if (g.act) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int a = g.bnat ^ f1::swz_c(e * NTA);
          const cplx<double> z = XH.ld(a);       // conj of n (v + i v_x)
          const double pv = z.x * inv_n, px = -z.y * inv_n;
          double c1, c2, c3;
          coef64(t + e * NTA, c1, c2, c3);
          XH.st(a, mk(c1 * pv + c2 * px, c2 * pv + c3 * px));
        }
      }
      split_h();
      f1::fft_smem<double, L>(XH, A.tw64);
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int k = g.mode(SL::b(q), SL::s(q));
          const double kk = kunit * (double)gm(k);
          const cplx<double> y = XH.ld(f1::swz(k));
          const cplx<double> ym = conj(XH.ld(f1::swz(mir(k))));
          const cplx<double> s = y * (1.0 - kk) + ym * (1.0 + kk);
          gq[q] = mk(0.5 * s.x, 0.5 * s.y);
        }
        if (ts) gN = mk(XH.ld(f1::swz(nl / 2)).x, 0.0);
      }
    };
    // r = b - G x0, p = A^{-1} r
    double rz;
    {
      cplx<double> gq[RP], gN = mk(0.0, 0.0);
      matvec(Xh, gq, gN);
      double loc = 0.0;
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int m = gm(g.mode(SL::b(q), SL::s(q)));
          const cplx<double> r = Bh[m] - gq[q];
          const double di = dinv64(m);
          Rh[m] = r;
          Ph[m] = r * di;
          loc += ((ts && q == 0) ? 1.0 : 2.0) * (r.x * r.x + r.y * r.y) * di;
        }
        if (ts) {
          const cplx<double> r = Bh[h] - gN;
          Rh[h] = r;
          Ph[h] = r * isig;
          loc += (r.x * r.x + r.y * r.y) * isig;
        }
      }
      rz = sum_d(loc);
    }
    while (sqrt(rz) > tol_abs) {
      if (iters >= maxit) {
        status = SGN_ERR_NOT_CONVERGED;
        break;
      }
      cplx<double> gq[RP], gN = mk(0.0, 0.0);
      matvec(Ph, gq, gN);
      double pq_loc = 0.0;
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const cplx<double> p = Ph[gm(g.mode(SL::b(q), SL::s(q)))];
          pq_loc += ((ts && q == 0) ? 1.0 : 2.0) * (p.x * gq[q].x + p.y * gq[q].y);
        }
        if (ts) pq_loc += Ph[h].x * gN.x;
      }
      const double pq = sum_d(pq_loc);
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double at = rz / pq;
      double rz_loc = 0.0;
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int m = gm(g.mode(SL::b(q), SL::s(q)));
          Xh[m] = Xh[m] + Ph[m] * at;
          const cplx<double> r = Rh[m] - gq[q] * at;
          Rh[m] = r;
          rz_loc += ((ts && q == 0) ? 1.0 : 2.0) * (r.x * r.x + r.y * r.y) * dinv64(m);
        }
        if (ts) {
          Xh[h] = Xh[h] + Ph[h] * at;
          const cplx<double> r = Rh[h] - gN * at;
          Rh[h] = r;
          rz_loc += (r.x * r.x + r.y * r.y) * isig;
        }
      }
      const double rz_new = sum_d(rz_loc);
      ++iters;
      if (!isfinite(rz_new)) {
        status = SGN_ERR_BREAKDOWN;
        break;
      }
      const double beta = rz_new / rz;
      rz = rz_new;
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int m = gm(g.mode(SL::b(q), SL::s(q)));
          Ph[m] = Rh[m] * dinv64(m) + Ph[m] * beta;
        }
        if (ts) Ph[h] = Rh[h] * isig + Ph[h] * beta;
      }
    }
    R.ratio = sqrt(rz) / bnorm;
    // x = F^{-1} x^ = conj(F(conj x^)) / n; with ux, the transform of Z = (1 - k) x^ (mirror
    // (1 + k) conj x^) instead, which gives x + i x_x
    to_real(Xh, ux != nullptr);
    if (g.act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const cplx<double> z = XH.ld(g.bnat ^ f1::swz_c(e * NTA));
        x[t + e * NTA] = z.x * inv_n;
        if (ux) static_cast<double*>(ux)[own + t + e * NTA] = -z.y * inv_n;
      }
    }
  } else {
    // ------------------------------------------------------------------ mixed precision
    const XBuf<float> XF(smem, nl);
    const XBuf<float> XFp = CL > 1 ? XBuf<float>(peer(smem), nl) : XF;
    const f1::TwF32 twf;
    cplx<float>* D = reinterpret_cast<cplx<float>*>(smem + SM::off_d);   // [RP + 1][NT]
    cplx<float>* Rr = reinterpret_cast<cplx<float>*>(smem + SM::off_r);  // [RP + 1][NT]
    const df inv_n(1.0f / (float)n, 0.0f);                                 // exact
    const float inv_nf = 1.0f / (float)n;
    const df one(1.0f, 0.0f), zero(0.0f, 0.0f);
    const df kh = num<df>(kunit);
    int refinements = 0;
    for (;;) {
      // ---- double-float residual r^ = b^ - (G x)^, writing the real-space x on the way
      cplx<float> rf[RP], rfN = mk(0.0f, 0.0f);
      {
        __syncthreads();                         // the previous correction d has been read
        if (g.act) {
          // conj(Z) with Z_m = (1 - k) x_m, Z_{n-m} = (1 + k) conj(x_m)
#pragma unroll
          for (int q = 0; q < RP; ++q) {
            const int kl = g.mode(SL::b(q), SL::s(q)), m = gm(kl);
            const df k = kh * df((float)m, 0.0f);
            const cplx<df> xv = Xh[m];
            if (ts && q == 0) {
              XH.st(0, mk(xv.x, zero));
            } else {
              XH.st(f1::swz(kl), conj(xv) * (one - k));
              XH.st(f1::swz(mir(kl)), xv * (one + k));
            }
          }
          if (ts) XH.st(f1::swz(nl / 2), mk(Xh[h].x, zero));
        }
        __syncthreads();
        f1::fft_smem<df, L>(XH, A.twdf);
        join_h();
        if (g.act) {
          // rolled: unrolled, the compiler hoists the 6 coefficient loads of every element
#pragma unroll 1
          for (int e = 0; e < E; ++e) {
            const int j = t + e * NTA;
            const int a = f1::swz(j);
            const cplx<df> z = XH.ld(a);         // conj of n (x + i x_x)
            const df pv = z.x * inv_n, px = -(z.y * inv_n);
            x[j] = to_f64(pv);
            if (ux) static_cast<df*>(ux)[own + j] = px;
            const df c1(cdf[j], cdf[3 * nl + j]), c2(cdf[nl + j], cdf[4 * nl + j]),
                c3(cdf[2 * nl + j], cdf[5 * nl + j]);
            XH.st(a, mk(c1 * pv + c2 * px, c2 * pv + c3 * px));
          }
        }
        split_h();
        f1::fft_smem<df, L>(XH, A.twdf);
        float rz_loc = 0.0f;
        if (g.act) {
#pragma unroll
          for (int q = 0; q < RP; ++q) {
            const int kl = g.mode(SL::b(q), SL::s(q)), m = gm(kl);
            const df k = kh * df((float)m, 0.0f);
            const cplx<df> y = XH.ld(f1::swz(kl));
            const cplx<df> ym = conj(XH.ld(f1::swz(mir(kl))));
            const cplx<df> s = y * (one - k) + ym * (one + k);
            const cplx<df> rr = Bh[m] - mk(half(s.x), half(s.y));
            rf[q] = mk(rr.x.hi + rr.x.lo, rr.y.hi + rr.y.lo);
            rz_loc += ((ts && q == 0) ? 1.0f : 2.0f) *
                      (rf[q].x * rf[q].x + rf[q].y * rf[q].y) * dinv(m);
          }
          if (ts) {
            const df rr = Bh[h].x - XH.ld(f1::swz(nl / 2)).x;
            rfN = mk(rr.hi + rr.lo, 0.0f);
            rz_loc += rfN.x * rfN.x * dN;
          }
        }
        // thread 0 decides the pass: converged, out of budget, or the next inner solve
        sum_f(rz_loc, slots, [&](float hi, float lo) {
          const double rz64 = (double)hi + (double)lo;
          const double nr = sqrt(rz64);
          const double ratio = nr / bnorm;
          ps.ratio = ratio;
          ps.go = 0;
          ps.status = status;
          if (ratio <= rtol || status != SGN_OK) return;
          if (refinements >= max_refine || iters >= maxit) {
            ps.status = SGN_ERR_NOT_CONVERGED;
            return;
          }
          const double tin =
              rtol_inner > 0.0 ? rtol_inner : fmin(0.1, fmax(1e-6, 0.3 * rtol / ratio));
          ps.scale = (float)(1.0 / nr);
          ps.unscale = df(nr);
          ps.tin2 = (float)(tin * tin);
          ps.go = 1;
        });
      }
      R.ratio = ps.ratio;
      status = ps.status;
      if (!ps.go) break;
      const float scale = ps.scale, tin2 = ps.tin2;
      const df unscale = ps.unscale;

      // ---- float32 PCG for G d = r / ||r||: p in registers, r, d and the preconditioner
      // symbol in thread-private shared slots (slot q of thread t at q NT + t)
      const int it_before = iters;
      int st_in = SGN_OK;
      {
        cplx<float> p[RP], pN = mk(0.0f, 0.0f);
        int it = iters;
        float loc = 0.0f;
        if (g.act) {
#pragma unroll
          for (int q = 0; q < RP; ++q) {
            const cplx<float> r = rf[q] * scale;
            p[q] = r * dinv(gm(g.mode(SL::b(q), SL::s(q))));
            loc += ((ts && q == 0) ? 1.0f : 2.0f) * (r.x * p[q].x + r.y * p[q].y);
            Rr[q * NT + t] = r;
            D[q * NT + t] = mk(0.0f, 0.0f);
          }
          if (ts) {
            const cplx<float> r = rfN * scale;
            pN = r * dN;
            loc += r.x * pN.x;
            Rr[RP * NT] = r;
            D[RP * NT] = mk(0.0f, 0.0f);
          }
        }
        sum_f(loc, slots + W, [&](float hi, float lo) {
          const float rz = hi + lo;
          sc.rz = rz;
          sc.state = (rz <= tin2) ? 1 : (it >= maxit ? 3 : 0);
        });
        for (;;) {
          const int state = sc.state;
          if (state != 0) {
            if (state == 3) st_in = SGN_ERR_NOT_CONVERGED;
            if (state == 2) st_in = SGN_ERR_BREAKDOWN;
            break;
          }
          cplx<float> v[E];
          if (g.act) {
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const float k = kf * (float)gm(g.mode(SL::b(q), SL::s(q)));
              if (ts && q == 0) {
                v[0] = mk(p[0].x, 0.0f);
              } else {
                v[SL::reg(q)] = p[q] * (1.0f - k);
                f1::mirror_set<L>(v, ts, SL::b(q), SL::s(q), conj(p[q]) * (1.0f + k));
              }
            }
            if (ts) v[HS] = mk(pN.x, 0.0f);
          }
          f1::fft_inv<float, L>(XF, v, g, twf);
          if constexpr (CL > 1)
            f1::cross<float, L, f1::kJoinInv>(XF, XFp, v, t, g.bnat, g.act, rk, nullptr);
          if (g.act) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int j = t + e * NTA;
              const float pv = v[e].x * inv_nf, px = v[e].y * inv_nf;
              const float et = eh[j], gx = eh[nl + j];
              const float e2 = et * et;
              const float c1 = fmaf(et * gx, gx, et), c2 = 0.5f * e2 * gx,
                          c3 = e2 * et * (1.0f / 3.0f);
              v[e] = mk(c1 * pv + c2 * px, c2 * pv + c3 * px);
            }
          }
          if constexpr (CL > 1)
            f1::cross<float, L, f1::kSplitFwd>(XF, XFp, v, t, g.bnat, g.act, rk, nullptr);
          f1::fft_fwd<float, L>(XF, v, g, twf);
          cplx<float> gq[RP], gN = mk(0.0f, 0.0f);
          float pq_loc = 0.0f;
          if (g.act) {
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const float k = kf * (float)gm(g.mode(SL::b(q), SL::s(q)));
              const cplx<float> y = v[SL::reg(q)];
              const cplx<float> ym = conj(f1::mirror_get<L>(v, ts, SL::b(q), SL::s(q)));
              const cplx<float> s = y * (1.0f - k) + ym * (1.0f + k);
              gq[q] = mk(0.5f * s.x, 0.5f * s.y);
              pq_loc += ((ts && q == 0) ? 1.0f : 2.0f) * (p[q].x * gq[q].x + p[q].y * gq[q].y);
            }
            if (ts) {
              gN = mk(v[HS].x, 0.0f);
              pq_loc += pN.x * gN.x;
            }
          }
          sum_f(pq_loc, slots, [&](float hi, float lo) {
            const float pq = hi + lo;
            if (!(pq > 0.0f) || !isfinite(pq)) sc.state = 2;
            else sc.alpha = sc.rz / pq;
          });
          if (sc.state == 2) {
            st_in = SGN_ERR_BREAKDOWN;
            break;
          }
          const float at = sc.alpha;
          float rz_loc = 0.0f;
          if (g.act) {
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const int o = q * NT + t;
              D[o] = D[o] + p[q] * at;
              const cplx<float> r = Rr[o] - gq[q] * at;
              Rr[o] = r;
              rz_loc += ((ts && q == 0) ? 1.0f : 2.0f) * (r.x * r.x + r.y * r.y) * dinv(gm(g.mode(SL::b(q), SL::s(q))));
            }
            if (ts) {
              D[RP * NT] = D[RP * NT] + pN * at;
              const cplx<float> r = Rr[RP * NT] - gN * at;
              Rr[RP * NT] = r;
              rz_loc += r.x * r.x * dN;
            }
          }
          ++it;
          sum_f(rz_loc, slots + W, [&](float hi, float lo) {
            const float rz_new = hi + lo;
            if (!isfinite(rz_new)) {
              sc.state = 2;
            } else {
              sc.beta = rz_new / sc.rz;
              sc.rz = rz_new;
              sc.state = (rz_new <= tin2) ? 1 : (it >= maxit ? 3 : 0);
            }
          });
          if (sc.state == 2) {
            st_in = SGN_ERR_BREAKDOWN;
            break;
          }
          const float beta = sc.beta;
          if (g.act) {
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const int o = q * NT + t;
              p[q] = Rr[o] * dinv(gm(g.mode(SL::b(q), SL::s(q)))) + p[q] * beta;
            }
            if (ts) pN = Rr[RP * NT] * dN + pN * beta;
          }
        }
        iters = it;
      }
      // A float32 breakdown after some progress only means float32 has resolved what it
      // can: keep the correction and let the next refinement pass decide.
      if (st_in == SGN_ERR_BREAKDOWN && iters == it_before) status = SGN_ERR_BREAKDOWN;
      ++refinements;
      // x^ += ||r|| d in double-float (each thread updates the modes of its own slots)
      if (g.act) {
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const int m = gm(g.mode(SL::b(q), SL::s(q)));
          const cplx<float> d = D[q * NT + t];
          const cplx<df> xv = Xh[m];
          Xh[m] = mk(xv.x + df(d.x, 0.0f) * unscale, xv.y + df(d.y, 0.0f) * unscale);
        }
        if (ts) {
          const cplx<float> d = D[RP * NT];
          const cplx<df> xv = Xh[h];
          Xh[h] = mk(xv.x + df(d.x, 0.0f) * unscale, xv.y);
        }
      }
    }
    R.refinements = refinements;
  }
  R.iters = iters;
  R.status = status;
  if (ts) A.rec[id] = R;
}

template <int L, bool MIXED, int CL>
__global__ void __launch_bounds__(Plan<L>::NT, Plan<L>::kMinBlocks)
    k_pcg1d(const __grid_constant__ PcgArgs A, int first) {
  pcg_body<L, MIXED, CL>(A, first, A.ux);
  // a CTA's shared memory must outlive the partner's last read of it
  if constexpr (CL > 1) cluster_sync();
}

}  // namespace pcg1d

template <int LG, int CL>
cudaError_t pcg1d_launch(const PcgArgs& a, int first, int num, cudaStream_t s) {
  static_assert(CL == 1 || CL == 2, "one CTA or a cluster of two per instance");
  static_assert(LG <= kSmemLog1d || CL == 2, "n = 16384 needs two CTAs");
  constexpr int L = LG - (CL - 1);          // points per CTA: 2^L
  using PL = f1::Plan<L>;
  const bool mixed = a.precision == SGN_PREC_MIXED;
  auto k = mixed ? pcg1d::k_pcg1d<L, true, CL> : pcg1d::k_pcg1d<L, false, CL>;
  const size_t sm = mixed ? pcg1d::SmemPcg<L>::mixed : pcg1d::SmemPcg<L>::fp64;
  cudaError_t e = d1::set_smem(k, sm);
  if (e) return e;
  return d1::launch_clustered<CL>(k, num, PL::NT, sm, s, a, first);
}

}  // namespace sgn
