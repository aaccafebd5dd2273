// a5 in 2d: the float32 inner PCG of the mixed solve (§3.2, Eq:PCGLinSyst, preconditioner A
// of §4) as ONE persistent cooperative launch per inner solve, for one or several 2d
// instances of the same grid size.
//
// Iteration (spectral space, vectors are half spectra [ny][H] of two components):
//   C1  column tiles: p = A^{-1} r + beta p (beta = 0 first), Hermitian projection of the
//       kx = 0 and kx = nx/2 columns, d^ = i kx p1^ + i ky p2^, column iFFT of (p1, p2, d)
//       into the three transform planes;
//   R   row pairs: C2R, the pointwise step of Def:MatrixM
//         w = eta (I + grad h grad h^T) p + eta^2/2 grad h d,  q = eta^2/2 grad h . p + eta^3/3 d,
//       and R2C back into the transform planes.  The same pass forms p.Gp in real space,
//       sum_x (p.w + d q) = (W p) . M (W p) with W p = (p, div p): Def:MatrixM writes
//       G = W^T M W, so this is the energy p.Gp exactly (Parseval); M is pointwise SPD, so
//       the sum is positive whenever p is not zero;
//   C2  column tiles: column FFT, G p^ = w^ - i k q^, x += alpha p, r -= alpha G p,
//       z = A^{-1} r and the partial sums of r.z.
// Grid-wide barriers separate the phases (three per iteration: the data exchange after C1
// and after R, which also publishes p.Gp for alpha, and the r.z sums after C2 for beta and
// the stopping test).  Every CTA sums the per-unit partials of each instance itself, in one
// fixed order, so all CTAs hold bitwise the same alpha, beta and decisions and leave the
// loop together; no scalar goes through the host.
//
// Data produced by other CTAs inside the launch (transform planes, Krylov vectors, partial
// sums) is read with ld.global.cg (L2, never a stale L1 line).  Each barrier waits at most
// kBarrierTimeoutNs; a CTA that gives up sets the error word, every CTA then leaves the
// loop at its next barrier, and the solve reports SGN_ERR_TIMEOUT.  The launch is
// cooperative, so every CTA of the grid is resident at once.
#include <cstdio>

#include "sgn_2d_dev.cuh"

namespace sgn {

using namespace d2;

namespace {

constexpr int kPNT = 512;                 // threads per CTA
constexpr int kPMaxE = 12;                // transform elements per thread: nb n <= 12 * 512
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

struct IScal {            // per-instance scalars, identical in every CTA
  double rz, tol, pq;
  float alpha, beta, sigf, alAf, isigf, kxu, kyu;
  int iters, cap, done, status;
};

// ---- transforms of the persistent kernel ------------------------------------------------
// Batched Stockham FFTs in shared memory with radix-8/4/2 stages held in registers, two
// buffers used in turn (one barrier per stage), twiddles from a 1024-entry table in shared
// memory, and one spare element after every 32 (pad) so the strided accesses of the stages
// spread over the banks.  Transform j of a batch lives at [j S, j S + pad_len(n)).
constexpr int kTwTab = 1024;                       // e^{-2 pi i m / 1024}, m < 1024
__device__ __forceinline__ int pad(int a) { return a + (a >> 5); }
__host__ __device__ constexpr int pad_len(int n) { return n + (n >> 5); }

__device__ __forceinline__ cplx<float> rot8(cplx<float> a, int q, bool inv) {
  // a * e^{-+2 pi i q / 8}, q = 1, 2, 3
  const float r = 0.70710678118654752f;
  if (q == 2) return inv ? mul_pi(a) : mul_mi(a);
  if (q == 1)
    return inv ? mk((a.x - a.y) * r, (a.x + a.y) * r) : mk((a.x + a.y) * r, (a.y - a.x) * r);
  return inv ? mk(-(a.x + a.y) * r, (a.x - a.y) * r) : mk((a.y - a.x) * r, -(a.x + a.y) * r);
}

// In-register DFT of R = 2, 4 or 8 points, output in natural order.
template <int R>
__device__ __forceinline__ void dft_reg(cplx<float>* x, bool inv) {
  if constexpr (R == 2) {
    const cplx<float> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else if constexpr (R == 4) {
    const cplx<float> s02 = x[0] + x[2], d02 = x[0] - x[2], s13 = x[1] + x[3], d13 = x[1] - x[3];
    const cplx<float> r13 = inv ? mul_pi(d13) : mul_mi(d13);
    x[0] = s02 + s13;
    x[1] = d02 + r13;
    x[2] = s02 - s13;
    x[3] = d02 - r13;
  } else {
    cplx<float> e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft_reg<4>(e, inv);
    dft_reg<4>(o, inv);
    x[0] = e[0] + o[0];
    x[4] = e[0] - o[0];
#pragma unroll
    for (int s = 1; s < 4; ++s) {
      const cplx<float> t = rot8(o[s], s, inv);
      x[s] = e[s] + t;
      x[s + 4] = e[s] - t;
    }
  }
}

// One radix-R stage at sub-transform length p (log2 lp) over nb transforms of length n:
// butterfly i of transform j reads src[i + r n/R], twiddles by w^{r k} (w = e^{-+2 pi i/(p R)},
// k = i mod p), and writes output s to dst[(i - k) R + k + s p].  MAXE bounds the elements a
// thread holds (nb n <= MAXE NT).
template <int NT, int MAXE, int R>
__device__ __forceinline__ void pstage(const cplx<float>* src, cplx<float>* dst, int log2n, int nb,
                                       int S, int lp, bool inv, const cplx<float>* tws) {
  constexpr int LR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  constexpr int MB = (MAXE + R - 1) / R;            // butterflies per thread
  const int lq = log2n - LR, q = 1 << lq;           // butterflies per transform
  const int tot = nb << lq;
  const int tsh = 10 - lp - LR;                     // table index of w^1: 2^tsh
  cplx<float> x[MB][R];
  int base[MB], out[MB];
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int g = threadIdx.x + b * NT;
    if (g < tot) {
      const int j = g >> lq, i = g & (q - 1), k = i & ((1 << lp) - 1);
      base[b] = j * S;
      out[b] = ((i - k) << LR) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[b][r] = src[base[b] + pad(i + r * q)];
      if (lp > 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const cplx<float> w = tws[(r * k) << tsh];
          x[b][r] = cmul_tw(x[b][r], w, inv);
        }
      }
      dft_reg<R>(x[b], inv);
    }
  }
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int g = threadIdx.x + b * NT;
    if (g < tot) {
#pragma unroll
      for (int s = 0; s < R; ++s) dst[base[b] + pad(out[b] + (s << lp))] = x[b][s];
    }
  }
  __syncthreads();
}

// Batched transform of nb sequences of length n = 2^log2n (8 <= n <= 1024) from buffer a,
// using b as the other buffer; returns the buffer that holds the result.  All NT threads
// call it; it returns after a barrier.
template <int NT, int MAXE>
__device__ __noinline__ cplx<float>* pfft(cplx<float>* a, cplx<float>* b, int log2n, int nb, int S,
                                          bool inv, const cplx<float>* tws) {
  const int ns = (log2n + 2) / 3;                   // stages of radix <= 8
  const int base = log2n / ns, extra = log2n - base * ns;
  int lp = 0;
  cplx<float>* src = a;
  cplx<float>* dst = b;
  for (int st = 0; st < ns; ++st) {
    const int bits = base + (st < extra ? 1 : 0);
    if (bits == 3) pstage<NT, MAXE, 8>(src, dst, log2n, nb, S, lp, inv, tws);
    else if (bits == 2) pstage<NT, MAXE, 4>(src, dst, log2n, nb, S, lp, inv, tws);
    else pstage<NT, MAXE, 2>(src, dst, log2n, nb, S, lp, inv, tws);
    lp += bits;
    cplx<float>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ cplx<float> ldcg(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ void stcg(cplx<float>* p, cplx<float> v) {
  __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}

// Grid-wide barrier on a monotone arrival counter: the k-th barrier of the launch waits for
// k * gridDim.x arrivals.  Returns true when the launch must stop (a wait gave up here or
// in another CTA).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned& target,
                                             int* s_stop) {
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned long long t0 = global_ns();
    int stop = 0;
    while (ld_acquire(bar) < target) {
      if (global_ns() - t0 > kBarrierTimeoutNs) {
        atomicExch(err, 1);
        stop = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *s_stop = stop | *reinterpret_cast<volatile int*>(err);
  }
  __syncthreads();
  return *s_stop != 0;
}

// Sum of the per-unit partials of every live instance (units [b U, b U + U)), each summed by
// one warp in a fixed order; fin(b, total) runs on one lane per instance.
template <typename Fin>
__device__ __forceinline__ void sum_units(const double* parts, int U, IScal* S, int B, Fin fin) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int b = w; b < B; b += kPNT / 32) {
    if (S[b].done) continue;
    double acc = 0.0;
    for (int i = l; i < U; i += 32) acc += __ldcg(parts + (long long)b * U + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (l == 0) fin(b, acc);
  }
  __syncthreads();
}

__device__ __forceinline__ float kx_of(const IScal& s, int c, int nx) {
  return c == (nx >> 1) ? 0.0f : s.kxu * (float)c;
}
__device__ __forceinline__ float ky_of(const IScal& s, int y, int ny) {
  return s.kyu * (float)wave_index(y, ny);
}
__device__ __forceinline__ void ainv(const IScal& s, float kx, float ky, cplx<float> r1,
                                     cplx<float> r2, cplx<float>& z1, cplx<float>& z2) {
  const float f = s.alAf * recip(s.sigf + s.alAf * (kx * kx + ky * ky));
  const cplx<float> kr = r1 * kx + r2 * ky;
  z1 = (r1 - kr * (f * kx)) * s.isigf;
  z2 = (r2 - kr * (f * ky)) * s.isigf;
}

// Block sum of float partials in double-float, returned as a double on thread 0.
__device__ __forceinline__ void block_part(float v, df* slot, double* out) {
  block_sum_df<kPNT>(v, slot, [&](float hi, float lo) { __stcg(out, (double)hi + (double)lo); });
}

// Shared memory of the kernel: the twiddle table, then two transform buffers A and B of
// max(3 TW, 3) transforms (column tiles: 3 planes x TW columns of ny; rows: 3 of nx).
struct PSmem {
  cplx<float>* tws;
  cplx<float>* A;
  cplx<float>* B;
};

// ---- C1: p update, projection, divergence, column iFFT --------------------------------
__device__ __forceinline__ void col_inverse(const PersistArgs2d& a, const PInst2d& I,
                                            const IScal& s, int c0, const PSmem& sm) {
  const int ny = a.ny, H = a.H, TW = a.tw, S = pad_len(ny), nx = a.nx;
  cplx<float>* buf = sm.A;
  const bool upd = s.beta != 0.0f;
  for (int e = threadIdx.x; e < TW * ny; e += kPNT) {
    const int y = e / TW, c = e - y * TW, col = c0 + c;
    cplx<float> p1 = mk(0.0f, 0.0f), p2 = p1;
    if (col < H) {
      const long long gi = (long long)y * H + col;
      const cplx<float> r1 = ldcg(I.r[0] + gi), r2 = ldcg(I.r[1] + gi);
      ainv(s, kx_of(s, col, nx), ky_of(s, y, ny), r1, r2, p1, p2);
      if (upd) {
        p1 = p1 + ldcg(I.p[0] + gi) * s.beta;
        p2 = p2 + ldcg(I.p[1] + gi) * s.beta;
      }
    }
    buf[(0 * TW + c) * S + pad(y)] = p1;
    buf[(1 * TW + c) * S + pad(y)] = p2;
  }
  __syncthreads();
  // the kx = 0 and kx = nx/2 columns of a real field are Hermitian in ky: project out the
  // rounding residue there before the packed C2R of the row pass could leak it
  for (int c = 0; c < TW; ++c) {
    const int col = c0 + c;
    if (col != 0 && col != (nx >> 1)) continue;
    for (int q = 0; q < 2; ++q) {
      cplx<float>* v = buf + (q * TW + c) * S;
      for (int y = threadIdx.x; y <= (ny >> 1); y += kPNT) {
        const int ym = (ny - y) & (ny - 1);
        const cplx<float> sm2 = v[pad(y)] + conj(v[pad(ym)]);
        const cplx<float> hm = mk(0.5f * sm2.x, 0.5f * sm2.y);
        v[pad(y)] = hm;
        v[pad(ym)] = conj(hm);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TW * ny; e += kPNT) {
    const int y = e / TW, c = e - y * TW, col = c0 + c;
    const cplx<float> p1 = buf[(0 * TW + c) * S + pad(y)], p2 = buf[(1 * TW + c) * S + pad(y)];
    cplx<float> d = mk(0.0f, 0.0f);
    if (col < H) {
      const long long gi = (long long)y * H + col;
      stcg(I.p[0] + gi, p1);
      stcg(I.p[1] + gi, p2);
      d = mul_ik(p1, kx_of(s, col, nx)) + mul_ik(p2, ky_of(s, y, ny));
    }
    buf[(2 * TW + c) * S + pad(y)] = d;
  }
  __syncthreads();
  const cplx<float>* o = pfft<kPNT, kPMaxE>(sm.A, sm.B, a.logny, 3 * TW, S, true, sm.tws);
  for (int e = threadIdx.x; e < TW * ny; e += kPNT) {
    const int y = e / TW, c = e - y * TW, col = c0 + c;
    if (col >= H) continue;
    const long long gi = (long long)y * H + col;
#pragma unroll
    for (int q = 0; q < 3; ++q) stcg(I.t[q] + gi, o[(q * TW + c) * S + pad(y)]);
  }
}

// ---- R: C2R, Def:MatrixM pointwise with the p.Gp partial, R2C --------------------------
__device__ __forceinline__ float row_matvec(const PersistArgs2d& a, const PInst2d& I, int y0,
                                            const PSmem& sm) {
  const int nx = a.nx, H = a.H, h = nx >> 1, S = pad_len(nx);
  const long long P = (long long)nx * a.ny;
  const int y1 = y0 + 1;
  // packed row r: (A, B) = (t0, t1) of row y0 (r = 0) or y1 (r = 1), (t2 of y0, t2 of y1)
  auto rowA = [&](int r) {
    return (r == 2 ? I.t[2] : I.t[0]) + (long long)(r == 1 ? y1 : y0) * H;
  };
  auto rowB = [&](int r) {
    return (r == 2 ? I.t[2] : I.t[1]) + (long long)(r == 0 ? y0 : y1) * H;
  };
  cplx<float>* z = sm.A;
  for (int e = threadIdx.x; e < 3 * nx; e += kPNT) {
    const int r = e / nx, m = e - r * nx;
    const int mm = m <= h ? m : nx - m;
    cplx<float> u = ldcg(rowA(r) + mm), v = ldcg(rowB(r) + mm);
    if (m > h) {
      u = conj(u);
      v = conj(v);
    }
    z[r * S + pad(m)] = mk(u.x - v.y, u.y + v.x);      // u + i v
  }
  __syncthreads();
  cplx<float>* w = pfft<kPNT, kPMaxE>(sm.A, sm.B, a.lognx, 3, S, true, sm.tws);
  const float inv = __int_as_float((127 - a.lognx - a.logny) << 23);   // 1 / (nx ny), exact
  const float third = 1.0f / 3.0f;
  float part = 0.0f;
  for (int x = threadIdx.x; x < nx; x += kPNT) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const long long j = (long long)(r ? y1 : y0) * nx + x;
      const cplx<float> pp = w[r * S + pad(x)];
      const cplx<float> dd = w[2 * S + pad(x)];
      const float p1 = pp.x * inv, p2 = pp.y * inv;
      const float d = (r ? dd.y : dd.x) * inv;
      const float e = I.ehh[j], hx = I.ehh[P + j], hy = I.ehh[2 * P + j];
      const float e2h = 0.5f * e * e;
      const float c11 = e * (1.0f + hx * hx), c12 = e * hx * hy, c22 = e * (1.0f + hy * hy);
      const float c13 = e2h * hx, c23 = e2h * hy, c33 = e * e * e * third;
      const float w1 = c11 * p1 + c12 * p2 + c13 * d;
      const float w2 = c12 * p1 + c22 * p2 + c23 * d;
      const float q = c13 * p1 + c23 * p2 + c33 * d;
      part += p1 * w1 + p2 * w2 + d * q;
      w[r * S + pad(x)] = mk(w1, w2);
      if (r) w[2 * S + pad(x)].y = q; else w[2 * S + pad(x)].x = q;
    }
  }
  __syncthreads();
  cplx<float>* other = w == sm.A ? sm.B : sm.A;
  const cplx<float>* Y = pfft<kPNT, kPMaxE>(w, other, a.lognx, 3, S, false, sm.tws);
  // R2C split of the three packed rows: A = (Y_m + conj Y_{n-m})/2, B = (Y_m - conj Y_{n-m})/(2i)
  for (int e = threadIdx.x; e < 3 * (h + 1); e += kPNT) {
    const int r = e / (h + 1), m = e - r * (h + 1);
    const cplx<float> yv = Y[r * S + pad(m)], yc = conj(Y[r * S + pad((nx - m) & (nx - 1))]);
    const cplx<float> sm2 = yv + yc, dm = mul_mi(yv - yc);
    stcg(const_cast<cplx<float>*>(rowA(r)) + m, mk(0.5f * sm2.x, 0.5f * sm2.y));
    stcg(const_cast<cplx<float>*>(rowB(r)) + m, mk(0.5f * dm.x, 0.5f * dm.y));
  }
  return part;
}

// ---- C2: column FFT, G p, x and r updates, r.z partial --------------------------------
__device__ __forceinline__ float col_forward_update(const PersistArgs2d& a, const PInst2d& I,
                                                    const IScal& s, int c0, const PSmem& sm) {
  const int ny = a.ny, H = a.H, TW = a.tw, S = pad_len(ny), nx = a.nx;
  cplx<float>* buf = sm.A;
  for (int e = threadIdx.x; e < TW * ny; e += kPNT) {
    const int y = e / TW, c = e - y * TW, col = c0 + c;
    const long long gi = (long long)y * H + col;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      buf[(q * TW + c) * S + pad(y)] = col < H ? ldcg(I.t[q] + gi) : mk(0.0f, 0.0f);
  }
  __syncthreads();
  const cplx<float>* o = pfft<kPNT, kPMaxE>(sm.A, sm.B, a.logny, 3 * TW, S, false, sm.tws);
  float part = 0.0f;
  const float al = s.alpha;
  for (int e = threadIdx.x; e < TW * ny; e += kPNT) {
    const int y = e / TW, c = e - y * TW, col = c0 + c;
    if (col >= H) continue;
    const long long gi = (long long)y * H + col;
    const float kx = kx_of(s, col, nx), ky = ky_of(s, y, ny);
    const cplx<float> qh = o[(2 * TW + c) * S + pad(y)];
    const cplx<float> g1 = o[(0 * TW + c) * S + pad(y)] - mul_ik(qh, kx);
    const cplx<float> g2 = o[(1 * TW + c) * S + pad(y)] - mul_ik(qh, ky);
    const cplx<float> p1 = ldcg(I.p[0] + gi), p2 = ldcg(I.p[1] + gi);
    stcg(I.x[0] + gi, ldcg(I.x[0] + gi) + p1 * al);
    stcg(I.x[1] + gi, ldcg(I.x[1] + gi) + p2 * al);
    const cplx<float> r1 = ldcg(I.r[0] + gi) - g1 * al, r2 = ldcg(I.r[1] + gi) - g2 * al;
    stcg(I.r[0] + gi, r1);
    stcg(I.r[1] + gi, r2);
    cplx<float> z1, z2;
    ainv(s, kx, ky, r1, r2, z1, z2);
    const float wgt = (col == 0 || col == (nx >> 1)) ? 1.0f : 2.0f;
    part += wgt * (r1.x * z1.x + r1.y * z1.y + r2.x * z2.x + r2.y * z2.y);
  }
  return part;
}

__global__ void __launch_bounds__(kPNT, 1) k2_pcg_persist(const __grid_constant__ PersistArgs2d a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ IScal S[kMaxBatch2d];
  __shared__ df slot[kPNT / 32];
  __shared__ int s_stop;
  PSmem sm;
  sm.tws = reinterpret_cast<cplx<float>*>(smem);
  sm.A = sm.tws + kTwTab;
  {
    const long long col = 3ll * a.tw * pad_len(a.ny), row = 3ll * pad_len(a.nx);
    sm.B = sm.A + (col > row ? col : row);
  }
  {
    // e^{-2 pi i m / 1024} from the 16384-entry float32 table
    const cplx<float>* tg = static_cast<const cplx<float>*>(a.tw32);
    for (int m = threadIdx.x; m < kTwTab; m += kPNT) sm.tws[m] = tg[m * (kTwiddleN / kTwTab)];
  }
  const int B = a.B, CU = a.col_units, RU = a.row_units;
  const long long P = (long long)a.nx * a.ny;
  for (int b = threadIdx.x; b < B; b += kPNT) {
    const Scal2d* sc = a.inst[b].sc;
    IScal s;
    s.rz = sc->rz;
    s.tol = sc->tol;
    s.pq = 0.0;
    s.alpha = 0.0f;
    s.beta = 0.0f;
    s.sigf = sc->sigf;
    s.alAf = sc->alphaAf;
    s.isigf = sc->isigf;
    s.kxu = (float)a.inst[b].kxu;
    s.kyu = (float)a.inst[b].kyu;
    s.iters = sc->iters;
    s.cap = sc->cap;
    s.done = sc->done;
    s.status = sc->status;
    S[b] = s;
  }
  if (threadIdx.x == 0) s_stop = 0;
  __syncthreads();
  unsigned target = 0;
  bool stop = false;
  for (;;) {
    int live = 0;
    for (int b = 0; b < B; ++b) live += S[b].done ? 0 : 1;
    if (!live) break;
    // ---- C1
    for (int u = blockIdx.x; u < B * CU; u += gridDim.x) {
      const int b = u / CU, tile = u - b * CU;
      if (S[b].done) continue;
      col_inverse(a, a.inst[b], S[b], tile * a.tw, sm);
      __syncthreads();
    }
    if ((stop = grid_barrier(a.bar, a.err, target, &s_stop))) break;
    // ---- R
    for (int u = blockIdx.x; u < B * RU; u += gridDim.x) {
      const int b = u / RU, pr = u - b * RU;
      if (S[b].done) continue;
      const float part = row_matvec(a, a.inst[b], 2 * pr, sm);
      block_part(part, slot, a.parts + (long long)b * RU + pr);
    }
    if ((stop = grid_barrier(a.bar, a.err, target, &s_stop))) break;
    // alpha = r.z / p.Gp (p.Gp in the half-spectrum units of r.z: P times the real sum)
    sum_units(a.parts, RU, S, B, [&](int b, double tot) {
      const double pq = tot * (double)P;
      if (!(pq > 0.0) || !isfinite(pq)) {
        S[b].status = SGN_ERR_BREAKDOWN;
        S[b].done = 1;
      } else {
        S[b].pq = pq;
        S[b].alpha = (float)(S[b].rz / pq);
      }
    });
    // ---- C2
    double* parts2 = a.parts + (long long)B * RU;
    for (int u = blockIdx.x; u < B * CU; u += gridDim.x) {
      const int b = u / CU, tile = u - b * CU;
      if (S[b].done) continue;
      const float part = col_forward_update(a, a.inst[b], S[b], tile * a.tw, sm);
      block_part(part, slot, parts2 + (long long)b * CU + tile);
    }
    if ((stop = grid_barrier(a.bar, a.err, target, &s_stop))) break;
    sum_units(parts2, CU, S, B, [&](int b, double rz) {
      IScal& s = S[b];
      s.iters += 1;
      if (!isfinite(rz)) {
        s.status = SGN_ERR_BREAKDOWN;
        s.done = 1;
      } else {
        s.beta = (float)(rz / s.rz);
        s.rz = rz;
        if (sqrt(rz) <= s.tol) {
          s.done = 1;
        } else if (s.iters >= s.cap) {
          s.status = SGN_ERR_NOT_CONVERGED;
          s.done = 1;
        }
      }
    });
  }
  if (blockIdx.x != 0) return;
  for (int b = threadIdx.x; b < B; b += kPNT) {
    Scal2d* sc = a.inst[b].sc;
    const IScal& s = S[b];
    sc->rz = s.rz;
    sc->iters = s.iters;
    sc->status = stop ? SGN_ERR_TIMEOUT : s.status;
    sc->done = 1;
    sc->alpha = (double)s.alpha;
    sc->alphaf = s.alpha;
    sc->beta = (double)s.beta;
    sc->betaf = s.beta;
  }
}

__global__ void k2_persist_arm(unsigned* bar, int* err) {
  *bar = 0u;
  *err = 0;
}

}  // namespace

// elements of one transform buffer: 3 tw columns of ny or 3 rows of nx, padded
long long persist2d_buf_elems(int nx, int ny, int tw) {
  const long long col = 3ll * tw * pad_len(ny), row = 3ll * pad_len(nx);
  return col > row ? col : row;
}

size_t persist2d_smem(int nx, int ny, int tw) {
  return sizeof(cplx<float>) * (kTwTab + 2 * persist2d_buf_elems(nx, ny, tw));
}

// Columns per tile: the widest of 4, 2, 1 whose three planes fit kPMaxE elements per thread
// and whose tiles still give every CTA of the grid a unit (four float32 columns fill a
// 32-byte sector of a row; a single instance of 512^2 takes one).
int persist2d_tile_width(int nx, int ny, int B, int grid) {
  const int H = nx / 2 + 1;
  for (int tw = 4; tw > 1; tw >>= 1)
    if (3 * tw * ny <= kPMaxE * kPNT && (long long)B * ((H + tw - 1) / tw) >= grid) return tw;
  return 1;
}

bool persist2d_tile_ok(int nx, int ny, int tw) {
  return tw >= 1 && tw <= 4 && 3 * tw * ny <= kPMaxE * kPNT;
}

// Resident CTAs of the persistent kernel on this device (one per SM: 512 threads of up to
// 128 registers), at most the largest phase's unit count.
cudaError_t persist2d_grid(int nx, int ny, int B, int* grid) {
  int tw_max = 4;
  while (tw_max > 1 && !persist2d_tile_ok(nx, ny, tw_max)) tw_max >>= 1;
  const size_t smem = persist2d_smem(nx, ny, tw_max);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k2_pcg_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(smem > 48 * 1024 ? smem : 48 * 1024))))
    return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_pcg_persist, kPNT, smem)))
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int H = nx / 2 + 1;
  const long long units = (long long)B * (H > ny / 2 ? H : ny / 2);
  long long g = (long long)per_sm * sms;
  if (units < g) g = units;
  *grid = (int)g;
  return cudaSuccess;
}

cudaError_t launch_pcg2d_persist(const PersistArgs2d& args, int grid, cudaStream_t s) {
  k2_persist_arm<<<1, 1, 0, s>>>(args.bar, args.err);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  const size_t smem = persist2d_smem(args.nx, args.ny, args.tw);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k2_pcg_persist, args);
}

}  // namespace sgn
