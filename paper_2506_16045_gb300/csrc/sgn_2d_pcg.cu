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
// sums) is read with ld.global.cg or copied to shared memory with cp.async.cg (both from L2,
// never a stale L1 line).  Where the shared memory allows (sides up to 512 with 128-thread
// groups, up to 1024 with 256-thread groups), the staged form gives each group a third
// buffer and issues all of a unit's input copies at once, so a unit waits for memory once
// instead of once per batch of rows.  Each barrier waits at most
// kBarrierTimeoutNs; a CTA that gives up sets the error word, every CTA then leaves the
// loop at its next barrier, and the solve reports SGN_ERR_TIMEOUT.  The launch is
// cooperative, so every CTA of the grid is resident at once.
#include <cstdio>

#include "sgn_2d_dev.cuh"

namespace sgn {

using namespace d2;

namespace {

constexpr int kPNT = 512;                 // threads per CTA
// Threads per group (GT): 128 (four groups per CTA, the default) or 256 (two groups, for
// solves with fewer units per phase than a grid's 128-thread groups).
constexpr int kRows = 1;                  // rows a thread loads per batch: with every phase
                                          // inlined, more would spill past 128 registers
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
// Twiddles per transform length n: for the stage of radix R at sub-length p, the block at
// offset p - 1 holds w^{r k} = e^{-2 pi i r k / (p R)} at (r - 1) p + k (r = 1..R-1, k < p), so
// the lanes of a warp read consecutive entries; the blocks of all stages take n - 1 entries.
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

// a * e^{-+2 pi i q / 16}, q = 1..9 (the twiddles inside a radix-16 butterfly)
__device__ __forceinline__ cplx<float> rot16(cplx<float> a, int q, bool inv) {
  constexpr float C[10] = {1.0f, 0.92387953251128676f, 0.70710678118654752f,
                           0.38268343236508977f, 0.0f, -0.38268343236508977f,
                           -0.70710678118654752f, -0.92387953251128676f, -1.0f,
                           -0.92387953251128676f};
  constexpr float Sn[10] = {0.0f, 0.38268343236508977f, 0.70710678118654752f,
                            0.92387953251128676f, 1.0f, 0.92387953251128676f,
                            0.70710678118654752f, 0.38268343236508977f, 0.0f,
                            -0.38268343236508977f};
  const float c = C[q], sn = inv ? Sn[q] : -Sn[q];       // e^{-+i pi q / 8}
  return mk(a.x * c - a.y * sn, a.x * sn + a.y * c);
}

// In-register DFT of R = 2, 4, 8 or 16 points, output in natural order.
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
  } else if constexpr (R == 16) {
    // 16 = 4 x 4: r = 4a + b, s = c + 4d; DFT4 over a, twiddle w16^{b c}, DFT4 over b
    cplx<float> A[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      cplx<float> v[4] = {x[b], x[4 + b], x[8 + b], x[12 + b]};
      dft_reg<4>(v, inv);
#pragma unroll
      for (int c = 0; c < 4; ++c) A[b][c] = (b && c) ? rot16(v[c], b * c, inv) : v[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      cplx<float> v[4] = {A[0][c], A[1][c], A[2][c], A[3][c]};
      dft_reg<4>(v, inv);
#pragma unroll
      for (int d = 0; d < 4; ++d) x[c + 4 * d] = v[d];
    }
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

// Barrier of one group of GT threads (named barrier g + 1; barrier 0 is __syncthreads).
template <int GT>
__device__ __forceinline__ void gsync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

// One radix-R stage at sub-transform length p (log2 lp) over nb transforms of length n, run
// by the GT threads of group g (thread t of the group): butterfly i of transform j reads
// src[i + r n/R], twiddles by w^{r k} (w = e^{-+2 pi i/(p R)}, k = i mod p), and writes output
// s to dst[(i - k) R + k + s p].  src and dst are different buffers, so each butterfly is
// written as soon as it is computed; the group barrier at the end orders the stages.
template <int R, int GT>
__device__ __forceinline__ void pstage(const cplx<float>* __restrict__ src,
                                       cplx<float>* __restrict__ dst, int log2n, int nb, int S,
                                       int lp, bool inv, const cplx<float>* __restrict__ tws,
                                       int t, int g) {
  constexpr int LR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
  const int lq = log2n - LR, q = 1 << lq;           // butterflies per transform
  const int tot = nb << lq;
  const int p0 = 1 << lp;
  // The padded addresses split into a per-butterfly part and per-stage constants that stay
  // out of the loop: pad(i + r q) = pad(i) + pad(r q) and, with k = i mod p,
  // pad((i - k) R + k + s p) = pad((i - k) R) + pad(k) + pad(s p) (q, p powers of two).
#pragma unroll 2
  for (int gi = t; gi < tot; gi += GT) {
    const int j = gi >> lq, i = gi & (q - 1), k = i & ((1 << lp) - 1);
    const cplx<float>* __restrict__ sb = src + j * S + pad(i);
    cplx<float>* __restrict__ db = dst + j * S + pad((i - k) << LR) + pad(k);
    cplx<float> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = sb[pad(r << lq)];
    if (lp > 0) {
      // w^r from the table for r = 1, 2, 4, 8; the other powers by one or two products
      const cplx<float>* tb = tws + p0 - 1 + k;
      cplx<float> w[R];
      w[1] = tb[0];
      if constexpr (R >= 4) {
        w[2] = tb[p0];
        w[3] = cmul(w[1], w[2]);
      }
      if constexpr (R >= 8) {
        w[4] = tb[3 * p0];
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
      }
      if constexpr (R >= 16) {
        w[8] = tb[7 * p0];
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul_tw(x[r], w[r], inv);
    }
    dft_reg<R>(x, inv);
#pragma unroll
    for (int s = 0; s < R; ++s) db[pad(s << lp)] = x[s];
  }
  gsync<GT>(g);
}

// Batched transform of nb sequences of length n = 2^log2n (8 <= n <= 1024) by group g, from
// buffer a with b as the other buffer; returns the buffer that holds the result.  Every
// thread of the group calls it; it returns after a group barrier.  The stages have radices
// up to 2^maxb (maxb = 4: radix 16, 3: radix 8), split as evenly as possible.
__device__ __forceinline__ int pfft_stages(int log2n, int maxb) { return (log2n + maxb - 1) / maxb; }

template <int GT>
__device__ __forceinline__ cplx<float>* pfft(cplx<float>* a, cplx<float>* b, int log2n, int nb, int S,
                                          bool inv, const cplx<float>* tws, int t, int g,
                                          int maxb) {
  const int ns = pfft_stages(log2n, maxb);
  const int base = log2n / ns, extra = log2n - base * ns;
  int lp = 0;
  cplx<float>* src = a;
  cplx<float>* dst = b;
  for (int st = 0; st < ns; ++st) {
    const int bits = base + (st < extra ? 1 : 0);
    if (bits == 4) pstage<16, GT>(src, dst, log2n, nb, S, lp, inv, tws, t, g);
    else if (bits == 3) pstage<8, GT>(src, dst, log2n, nb, S, lp, inv, tws, t, g);
    else if (bits == 2) pstage<4, GT>(src, dst, log2n, nb, S, lp, inv, tws, t, g);
    else pstage<2, GT>(src, dst, log2n, nb, S, lp, inv, tws, t, g);
    lp += bits;
    cplx<float>* tmp = src;
    src = dst;
    dst = tmp;
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
// Asynchronous 16-byte copy global -> shared that bypasses L1 (cp.async.cg), and the wait
// for all of this thread's copies; both addresses 16-byte aligned.
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
    for (int i0 = 0; i0 < U; i0 += 8 * 32) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = i0 + l + 32 * k;
        v[k] = i < U ? __ldcg(parts + (long long)b * U + i) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) acc += v[k];
    }
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

// Sum of the float partials of group g in double-float, stored as a double to `out` by the
// group's thread 0 (warp shuffles, then the group's four warp totals in order).
template <int GT>
__device__ __forceinline__ void group_part(float v, df* slot, double* out, int t, int g) {
  df a(v, 0.0f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df b(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    a = a + b;
  }
  if ((t & 31) == 0) slot[g * (GT / 32) + (t >> 5)] = a;
  gsync<GT>(g);
  if (t == 0) {
    df r = slot[g * (GT / 32)];
#pragma unroll
    for (int w = 1; w < GT / 32; ++w) r = r + slot[g * (GT / 32) + w];
    __stcg(out, (double)r.hi + (double)r.lo);
  }
  gsync<GT>(g);
}

// Shared memory of the kernel: the twiddle table, then per group two transform buffers of
// three columns of ny or three rows of nx (padded) and, in the staged form, a third buffer
// C that receives a unit's global inputs by asynchronous copies.
struct PSmem {
  cplx<float>* twx;     // twiddles of length nx
  cplx<float>* twy;     // of length ny (the same table when ny = nx)
  cplx<float>* A;       // this group's buffers
  cplx<float>* B;
  cplx<float>* C;       // staged form only
};

// Sizes in complex float32 entries, both even (16-byte aligned buffers).  A and B each hold
// three padded transforms; staged, B also takes the raw row pairs of a row unit (6 (nx/2 + 1)
// entries).  C holds the largest unit input: six columns of ny (the C2 update vectors) or
// three planes' float32 coefficients of two rows (3 nx entries).
__host__ __device__ inline int persist_be(int nx, int ny, bool stg) {
  int be = 3 * pad_len(nx > ny ? nx : ny);
  if (stg && be < 6 * (nx / 2 + 1)) be = 6 * (nx / 2 + 1);
  return (be + 1) & ~1;
}
__host__ __device__ inline int persist_bc(int nx, int ny, bool stg) {
  if (!stg) return 0;
  return 6 * ny > 3 * nx ? 6 * ny : 3 * nx;
}

// ---- C1: p update, projection, divergence, column iFFT (column c, group g) -------------
// The solve's vectors and transform planes are column-major, [H][ny]: a column is contiguous.
template <bool STG, int GT>
__device__ __forceinline__ void col_inverse(const PersistArgs2d& a, const PInst2d& I,
                                         const IScal& s, int c, const PSmem& sm, int t, int g) {
  const int ny = a.ny, S = pad_len(ny), nx = a.nx;
  const long long cb = (long long)c * ny;
  cplx<float>* buf = sm.A;
  const bool upd = s.beta != 0.0f;
  const float kx = kx_of(s, c, nx);
  const cplx<float>* __restrict__ r0 = I.r[0] + cb;
  const cplx<float>* __restrict__ r1p = I.r[1] + cb;
  cplx<float>* __restrict__ p0 = I.p[0] + cb;
  cplx<float>* __restrict__ p1p = I.p[1] + cb;
  if constexpr (STG) {
    // every load of the unit in flight at once: r1, r2 (and p1, p2 when beta != 0) into C as
    // 16-byte copies, then p = A^{-1} r + beta p from shared memory
    cplx<float>* Cb = sm.C;
    const int lch = a.logny - 1, nch = (upd ? 4 : 2) << lch;
    for (int i = t; i < nch; i += GT) {
      const int q = i >> lch, e = (i - (q << lch)) << 1;
      const cplx<float>* src = q == 0 ? r0 : (q == 1 ? r1p : (q == 2 ? p0 : p1p));
      cp16(Cb + q * ny + e, src + e);
    }
    cp_wait_all();
    gsync<GT>(g);
    for (int y = t; y < ny; y += GT) {
      cplx<float> p1, p2;
      ainv(s, kx, ky_of(s, y, ny), Cb[y], Cb[ny + y], p1, p2);
      if (upd) {
        p1 = p1 + Cb[2 * ny + y] * s.beta;
        p2 = p2 + Cb[3 * ny + y] * s.beta;
      }
      buf[pad(y)] = p1;
      buf[S + pad(y)] = p2;
    }
  } else {
  // the column's loads first (kRows rows per thread in flight), then the shared stores
  for (int y0 = 0; y0 < ny; y0 += kRows * GT) {
    cplx<float> r1[kRows], r2[kRows], q1[kRows], q2[kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
        r1[k] = ldcg(r0 + y);
        r2[k] = ldcg(r1p + y);
        if (upd) {
          q1[k] = ldcg(p0 + y);
          q2[k] = ldcg(p1p + y);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
        cplx<float> p1, p2;
        ainv(s, kx, ky_of(s, y, ny), r1[k], r2[k], p1, p2);
        if (upd) {
          p1 = p1 + q1[k] * s.beta;
          p2 = p2 + q2[k] * s.beta;
        }
        buf[pad(y)] = p1;
        buf[S + pad(y)] = p2;
      }
    }
  }
  }
  gsync<GT>(g);
  // the kx = 0 and kx = nx/2 columns of a real field are Hermitian in ky: project out the
  // rounding residue there before the packed C2R of the row pass could leak it
  if (c == 0 || c == (nx >> 1)) {
    for (int q = 0; q < 2; ++q) {
      cplx<float>* v = buf + q * S;
      for (int y = t; y <= (ny >> 1); y += GT) {
        const int ym = (ny - y) & (ny - 1);
        const cplx<float> sm2 = v[pad(y)] + conj(v[pad(ym)]);
        const cplx<float> hm = mk(0.5f * sm2.x, 0.5f * sm2.y);
        v[pad(y)] = hm;
        v[pad(ym)] = conj(hm);
      }
    }
    gsync<GT>(g);
  }
  for (int y = t; y < ny; y += GT) {
    const cplx<float> p1 = buf[pad(y)], p2 = buf[S + pad(y)];
    stcg(p0 + y, p1);
    stcg(p1p + y, p2);
    buf[2 * S + pad(y)] = mul_ik(p1, kx) + mul_ik(p2, ky_of(s, y, ny));
  }
  gsync<GT>(g);
  const cplx<float>* o = pfft<GT>(sm.A, sm.B, a.logny, 3, S, true, sm.twy, t, g, a.maxb);
  for (int y = t; y < ny; y += GT) {
#pragma unroll
    for (int q = 0; q < 3; ++q) stcg(I.t[q] + cb + y, o[q * S + pad(y)]);
  }
}

// ---- R: C2R, Def:MatrixM pointwise with the p.Gp partial, R2C (row pair y0, group g) -----
template <bool STG, int GT>
__device__ __forceinline__ float row_matvec(const PersistArgs2d& a, const PInst2d& I, int y0,
                                            const PSmem& sm, int t, int g) {
  const int nx = a.nx, h = nx >> 1, S = pad_len(nx);
  const long long P = (long long)nx * a.ny;
  const int y1 = y0 + 1;
  // Column m of the transform planes holds rows y0 and y1 side by side (16 bytes): one load
  // per plane gives packed row 0 (t0, t1 of y0), row 1 (t0, t1 of y1) and row 2 (t2 of y0,
  // t2 of y1) at mode m; modes above nx/2 are the conjugates of nx - m.
  cplx<float>* z = sm.A;
  auto pair_ld = [&](int q, int m) {
    return __ldcg(reinterpret_cast<const float4*>(I.t[q] + (long long)m * a.ny + y0));
  };
  auto put = [&](int m, cplx<float> u0, cplx<float> v0, cplx<float> u1, cplx<float> v1,
                 cplx<float> u2, cplx<float> v2) {
    z[pad(m)] = mk(u0.x - v0.y, u0.y + v0.x);          // u + i v
    z[S + pad(m)] = mk(u1.x - v1.y, u1.y + v1.x);
    z[2 * S + pad(m)] = mk(u2.x - v2.y, u2.y + v2.x);
  };
  // staged: the raw row pairs of the three planes go to B (16-byte entries [q (h + 1) + m])
  // and the six coefficient rows (eta, h_x, h_y of rows y0, y1) to C ([(2 j + r) nx + x]),
  // all copies in flight at once; the packing then reads shared memory
  const float* ef = reinterpret_cast<const float*>(sm.C);
  if constexpr (STG) {
    float4* raw = reinterpret_cast<float4*>(sm.B);
    const int hp = h + 1;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      for (int m = t; m <= h; m += GT) cp16(raw + q * hp + m, I.t[q] + (long long)m * a.ny + y0);
    float* ed = reinterpret_cast<float*>(sm.C);
    const int lc = a.lognx - 2, nch = 6 << lc;
    for (int i = t; i < nch; i += GT) {
      const int row = i >> lc, e = (i - (row << lc)) << 2, j = row >> 1, r = row & 1;
      cp16(ed + row * nx + e, I.ehh + j * P + (long long)(y0 + r) * nx + e);
    }
    cp_wait_all();
    gsync<GT>(g);
    for (int m = t; m <= h; m += GT) {
      const float4 A0 = raw[m], A1 = raw[hp + m], A2 = raw[2 * hp + m];
      const cplx<float> a0 = mk(A0.x, A0.y), a1 = mk(A0.z, A0.w);
      const cplx<float> b0 = mk(A1.x, A1.y), b1 = mk(A1.z, A1.w);
      const cplx<float> d0 = mk(A2.x, A2.y), d1 = mk(A2.z, A2.w);
      put(m, a0, b0, a1, b1, d0, d1);
      if (m > 0 && m < h) put(nx - m, conj(a0), conj(b0), conj(a1), conj(b1), conj(d0), conj(d1));
    }
  } else
  for (int m0 = 0; m0 <= h; m0 += kRows * GT) {
    float4 A0[kRows], A1[kRows], A2[kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int m = m0 + t + k * GT;
      if (m <= h) {
        A0[k] = pair_ld(0, m);
        A1[k] = pair_ld(1, m);
        A2[k] = pair_ld(2, m);
      }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int m = m0 + t + k * GT;
      if (m <= h) {
        // t0 = (p1(y0), p1(y1)), t1 = (p2(y0), p2(y1)), t2 = (d(y0), d(y1))
        const cplx<float> a0 = mk(A0[k].x, A0[k].y), a1 = mk(A0[k].z, A0[k].w);
        const cplx<float> b0 = mk(A1[k].x, A1[k].y), b1 = mk(A1[k].z, A1[k].w);
        const cplx<float> d0 = mk(A2[k].x, A2[k].y), d1 = mk(A2[k].z, A2[k].w);
        put(m, a0, b0, a1, b1, d0, d1);
        if (m > 0 && m < h) put(nx - m, conj(a0), conj(b0), conj(a1), conj(b1), conj(d0), conj(d1));
      }
    }
  }
  gsync<GT>(g);
  cplx<float>* w = pfft<GT>(sm.A, sm.B, a.lognx, 3, S, true, sm.twx, t, g, a.maxb);
  const float inv = __int_as_float((127 - a.lognx - a.logny) << 23);   // 1 / (nx ny), exact
  const float third = 1.0f / 3.0f;
  float part = 0.0f;
  for (int x0 = 0; x0 < nx; x0 += kRows * GT) {
    // eta, h_x, h_y of both rows for kRows points per thread, loaded before use
    float ev[kRows][2], hxv[kRows][2], hyv[kRows][2];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int x = x0 + t + k * GT;
      if (x < nx) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if constexpr (STG) {
            ev[k][r] = ef[r * nx + x];
            hxv[k][r] = ef[(2 + r) * nx + x];
            hyv[k][r] = ef[(4 + r) * nx + x];
          } else {
            const long long j = (long long)(r ? y1 : y0) * nx + x;
            ev[k][r] = I.ehh[j];
            hxv[k][r] = I.ehh[P + j];
            hyv[k][r] = I.ehh[2 * P + j];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int x = x0 + t + k * GT;
      if (x >= nx) continue;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const cplx<float> pp = w[r * S + pad(x)];
        const cplx<float> dd = w[2 * S + pad(x)];
        const float p1 = pp.x * inv, p2 = pp.y * inv;
        const float d = (r ? dd.y : dd.x) * inv;
        const float e = ev[k][r], hx = hxv[k][r], hy = hyv[k][r];
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
  }
  gsync<GT>(g);
  cplx<float>* other = w == sm.A ? sm.B : sm.A;
  const cplx<float>* Y = pfft<GT>(w, other, a.lognx, 3, S, false, sm.twx, t, g, a.maxb);
  // R2C split of the three packed rows, A = (Y_m + conj Y_{n-m})/2, B = (Y_m - conj Y_{n-m})/(2i),
  // stored back as row pairs of columns m: t0 = (A_0, A_1), t1 = (B_0, B_1), t2 = (A_2, B_2)
  for (int m = t; m <= h; m += GT) {
    cplx<float> A_[3], B_[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const cplx<float> yv = Y[r * S + pad(m)], yc = conj(Y[r * S + pad((nx - m) & (nx - 1))]);
      const cplx<float> sm2 = yv + yc, dm = mul_mi(yv - yc);
      A_[r] = mk(0.5f * sm2.x, 0.5f * sm2.y);
      B_[r] = mk(0.5f * dm.x, 0.5f * dm.y);
    }
    const long long o = (long long)m * a.ny + y0;
    __stcg(reinterpret_cast<float4*>(I.t[0] + o), make_float4(A_[0].x, A_[0].y, A_[1].x, A_[1].y));
    __stcg(reinterpret_cast<float4*>(I.t[1] + o), make_float4(B_[0].x, B_[0].y, B_[1].x, B_[1].y));
    __stcg(reinterpret_cast<float4*>(I.t[2] + o), make_float4(A_[2].x, A_[2].y, B_[2].x, B_[2].y));
  }
  return part;
}

// ---- C2: column FFT, G p, x and r updates, r.z partial (column c, group g) ---------------
template <bool STG, int GT>
__device__ __forceinline__ float col_forward_update(const PersistArgs2d& a, const PInst2d& I,
                                                    const IScal& s, int c, const PSmem& sm,
                                                    int t, int g) {
  const int ny = a.ny, S = pad_len(ny), nx = a.nx;
  const long long cb = (long long)c * ny;
  cplx<float>* buf = sm.A;
  const cplx<float>* Cb = sm.C;
  if constexpr (STG) {
    // every load of the unit in flight at once: the three plane columns to B (unpadded) and
    // p1, p2, x1, x2, r1, r2 to C, as 16-byte copies; then the planes are spread into A's
    // padded transform layout
    cplx<float>* Bb = sm.B;
    cplx<float>* Cw = sm.C;
    const int lch = a.logny - 1;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      for (int e = 2 * t; e < ny; e += 2 * GT) cp16(Bb + q * ny + e, I.t[q] + cb + e);
    const int nch = 6 << lch;
    for (int i = t; i < nch; i += GT) {
      const int q = i >> lch, e = (i - (q << lch)) << 1;
      const cplx<float>* src = q < 2 ? I.p[q] : (q < 4 ? I.x[q - 2] : I.r[q - 4]);
      cp16(Cw + q * ny + e, src + cb + e);
    }
    cp_wait_all();
    gsync<GT>(g);
    for (int y = t; y < ny; y += GT) {
#pragma unroll
      for (int q = 0; q < 3; ++q) buf[q * S + pad(y)] = Bb[q * ny + y];
    }
  } else
  for (int y0 = 0; y0 < ny; y0 += kRows * GT) {
    cplx<float> v[3][kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q][k] = ldcg(I.t[q] + cb + y);
      }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
#pragma unroll
        for (int q = 0; q < 3; ++q) buf[q * S + pad(y)] = v[q][k];
      }
    }
  }
  gsync<GT>(g);
  const cplx<float>* o = pfft<GT>(sm.A, sm.B, a.logny, 3, S, false, sm.twy, t, g, a.maxb);
  float part = 0.0f;
  const float al = s.alpha;
  const float kx = kx_of(s, c, nx);
  const float wgt = (c == 0 || c == (nx >> 1)) ? 1.0f : 2.0f;
  cplx<float>* __restrict__ X0 = I.x[0] + cb;
  cplx<float>* __restrict__ X1 = I.x[1] + cb;
  cplx<float>* __restrict__ R0 = I.r[0] + cb;
  cplx<float>* __restrict__ R1 = I.r[1] + cb;
  const cplx<float>* __restrict__ P0 = I.p[0] + cb;
  const cplx<float>* __restrict__ P1 = I.p[1] + cb;
  constexpr int KU = kRows;         // rows per batch of the update (six loads each)
  for (int y0 = 0; y0 < ny; y0 += KU * GT) {
    cplx<float> p1[KU], p2[KU], x1[KU], x2[KU], r1[KU], r2[KU];
#pragma unroll
    for (int k = 0; k < KU; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
        if constexpr (STG) {
          p1[k] = Cb[y];
          p2[k] = Cb[ny + y];
          x1[k] = Cb[2 * ny + y];
          x2[k] = Cb[3 * ny + y];
          r1[k] = Cb[4 * ny + y];
          r2[k] = Cb[5 * ny + y];
        } else {
          p1[k] = ldcg(P0 + y);
          p2[k] = ldcg(P1 + y);
          x1[k] = ldcg(X0 + y);
          x2[k] = ldcg(X1 + y);
          r1[k] = ldcg(R0 + y);
          r2[k] = ldcg(R1 + y);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KU; ++k) {
      const int y = y0 + t + k * GT;
      if (y < ny) {
        const float ky = ky_of(s, y, ny);
        const cplx<float> qh = o[2 * S + pad(y)];
        const cplx<float> g1 = o[pad(y)] - mul_ik(qh, kx);
        const cplx<float> g2 = o[S + pad(y)] - mul_ik(qh, ky);
        stcg(X0 + y, x1[k] + p1[k] * al);
        stcg(X1 + y, x2[k] + p2[k] * al);
        const cplx<float> nr1 = r1[k] - g1 * al, nr2 = r2[k] - g2 * al;
        stcg(R0 + y, nr1);
        stcg(R1 + y, nr2);
        cplx<float> z1, z2;
        ainv(s, kx, ky, nr1, nr2, z1, z2);
        part += wgt * (nr1.x * z1.x + nr1.y * z1.y + nr2.x * z2.x + nr2.y * z2.y);
      }
    }
  }
  return part;
}

// STG: the staged form (a third shared buffer per group takes each unit's global inputs
// by asynchronous copies, all in flight at once); otherwise loads go through registers.
template <bool STG, int GT>
__global__ void __launch_bounds__(kPNT, 1) k2_pcg_persist(const __grid_constant__ PersistArgs2d a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ IScal S[kMaxBatch2d];
  __shared__ df slot[kPNT / 32];        // the groups' warp totals
  __shared__ int s_stop;
  // thread t of group g; the group's buffers after the twiddle table
  const int g = threadIdx.x / GT, t = threadIdx.x - g * GT;
  const int be = persist_be(a.nx, a.ny, STG), bc = persist_bc(a.nx, a.ny, STG);
  const int ntw = a.nx + (a.ny == a.nx ? 0 : a.ny);
  PSmem sm;
  sm.twx = reinterpret_cast<cplx<float>*>(smem);
  sm.twy = a.ny == a.nx ? sm.twx : sm.twx + a.nx;
  sm.A = sm.twx + ntw + (2 * be + bc) * g;
  sm.B = sm.A + be;
  sm.C = sm.B + be;
  {
    // the stage tables of both lengths from the 16384-entry float32 table e^{-2 pi i m / 16384}
    const cplx<float>* tg = static_cast<const cplx<float>*>(a.tw32);
    for (int which = 0; which < (a.ny == a.nx ? 1 : 2); ++which) {
      const int log2n = which ? a.logny : a.lognx;
      cplx<float>* tab = which ? sm.twy : sm.twx;
      const int ns = pfft_stages(log2n, a.maxb), base = log2n / ns, extra = log2n - base * ns;
      int lp = 0;
      for (int st = 0; st < ns; ++st) {
        const int bits = base + (st < extra ? 1 : 0), R = 1 << bits, p0 = 1 << lp;
        for (int e = threadIdx.x; e < (R - 1) * p0; e += kPNT) {
          const int r = 1 + e / p0, k = e - (r - 1) * p0;
          tab[p0 - 1 + e] = tg[(r * k) << (kTwiddleLog2 - lp - bits)];
        }
        lp += bits;
      }
    }
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
    // Units go to the groups of the grid in turn, group-major (slot = group * grid + CTA),
    // so a phase with fewer units than slots still spreads over every SM; adjacent columns
    // (which share the 32-byte sectors of every row) are in flight together.
    const int slot0 = g * gridDim.x + blockIdx.x, nslots = gridDim.x * (kPNT / GT);
    // ---- C1
    for (int u = slot0; u < B * CU; u += nslots) {
      const int b = u / CU, c = u - b * CU;
      if (S[b].done) continue;
      col_inverse<STG, GT>(a, a.inst[b], S[b], c, sm, t, g);
      gsync<GT>(g);
    }
    if ((stop = grid_barrier(a.bar, a.err, target, &s_stop))) break;
    // ---- R
    for (int u = slot0; u < B * RU; u += nslots) {
      const int b = u / RU, pr = u - b * RU;
      if (S[b].done) continue;
      const float part = row_matvec<STG, GT>(a, a.inst[b], 2 * pr, sm, t, g);
      group_part<GT>(part, slot, a.parts + (long long)b * RU + pr, t, g);
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
    for (int u = slot0; u < B * CU; u += nslots) {
      const int b = u / CU, c = u - b * CU;
      if (S[b].done) continue;
      const float part = col_forward_update<STG, GT>(a, a.inst[b], S[b], c, sm, t, g);
      group_part<GT>(part, slot, parts2 + (long long)b * CU + c, t, g);
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

// Shared memory: the twiddle tables and, per group of gt threads, two buffers of three
// padded transforms (and the staged form's input buffer).
static size_t persist_smem(int nx, int ny, bool stg, int gt) {
  const long long ntw = nx + (ny == nx ? 0 : ny);
  const long long per = 2ll * persist_be(nx, ny, stg) + persist_bc(nx, ny, stg);
  return sizeof(cplx<float>) * (ntw + per * (kPNT / gt));
}

using PersistKernel = void (*)(PersistArgs2d);
static PersistKernel persist_kernel(bool stg, int gt) {
  if (gt == 256) return stg ? k2_pcg_persist<true, 256> : k2_pcg_persist<false, 256>;
  return stg ? k2_pcg_persist<true, 128> : k2_pcg_persist<false, 128>;
}

// The staged form runs where its shared memory (with the kernel's static part) fits one
// CTA on this device: with 128-thread groups sides up to 512, with 256-thread groups up to
// 1024, on a 227 KB part.
static cudaError_t persist_staged(int nx, int ny, int gt, bool* stg) {
  int dev = 0, optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, persist_kernel(true, gt)))) return e;
  *stg = fa.sharedSizeBytes + persist_smem(nx, ny, true, gt) <= (size_t)optin;
  return cudaSuccess;
}

// Threads per unit: the layout's choice, else 256 when the largest phase has at most one
// unit per 256-thread group of the grid (each unit then finishes in about half the time and
// no group waits for a second round), else 128.
static int persist_gt(const PersistArgs2d& a, int grid) {
  if (a.gt == 128 || a.gt == 256) return a.gt;
  const long long units = (long long)a.B * (a.col_units > a.row_units ? a.col_units : a.row_units);
  return units <= 2ll * grid ? 256 : 128;
}

// A column unit is one half-spectrum column (each group transforms three planes of it).
int persist2d_tile_width(int nx, int ny, int B, int grid) {
  (void)nx;
  (void)ny;
  (void)B;
  (void)grid;
  return 1;
}

bool persist2d_tile_ok(int nx, int ny, int tw) {
  (void)nx;
  (void)ny;
  return tw == 1;
}

// Resident CTAs of the persistent kernel on this device (one per SM: 512 threads of up to
// 128 registers), at most the largest phase's unit count.
cudaError_t persist2d_grid(int nx, int ny, int B, int* grid) {
  cudaError_t e;
  PersistKernel k128 = nullptr;
  size_t smem128 = 0;
  for (int gt : {128, 256}) {
    bool stg = false;
    if ((e = persist_staged(nx, ny, gt, &stg))) return e;
    const size_t smem = persist_smem(nx, ny, stg, gt);
    if ((e = raise_smem(persist_kernel(stg, gt), smem))) return e;
    if (gt == 128) {
      k128 = persist_kernel(stg, gt);
      smem128 = smem;
    }
  }
  // the 128-thread form holds the most shared memory: its residency bounds both forms
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k128, kPNT, smem128))) return e;
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
  const int gt = persist_gt(args, grid);
  bool stg = false;
  if ((e = persist_staged(args.nx, args.ny, gt, &stg))) return e;
  const size_t smem = persist_smem(args.nx, args.ny, stg, gt);
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
  return cudaLaunchKernelEx(&cfg, persist_kernel(stg, gt), args);
}

}  // namespace sgn
