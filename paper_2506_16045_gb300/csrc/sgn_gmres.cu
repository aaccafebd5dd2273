// Restarted GMRES(m) for G_{eta,h} x = b with right preconditioning by the constant-
// coefficient A of §4: the Krylov option besides PCG.  G is SPD, so PCG (§3.2) is the
// method of the paper and the cheaper one; GMRES serves operators that lose symmetry (a
// non-symmetric discretisation or the non-constraint form) and as a cross-check of PCG.
//
// Inner product.  The Arnoldi process runs in <u, v> = u . A^{-1} v, so every iterate
// minimises sqrt(r.A^{-1}r), the residual measure of the PCG stopping rule.  In the
// Euclidean norm a fine grid's residual has a rounding floor near eps ||G|| (G grows like
// eta^3 k^2 / 3: about 1e-8 relative at n = 8192 on L = 1), which A^{-1} damps.  The basis
// is kept twice, V and Z = A^{-1} V: the next matvec is G Z_j and needs no A-solve, the one
// A-solve per step is t = A^{-1} w, and the Gram-Schmidt updates carry t along with w.
//
// Design.  Every instance of a layout runs its own GMRES on its own segment of the packed
// vectors, all in one set of launches per Arnoldi step:
//   w = G Z_j, t = A^{-1} w        the float64 operator kernels of the library
//   h = Z^T w, w -= V h, t -= Z h  classical Gram-Schmidt with one reorthogonalisation (twice):
//                                 two block-parallel passes over the basis instead of j + 1
//                                 dependent ones; the second restores the orthogonality that
//                                 one classical pass loses
//   sqrt(w.t), Givens rotations   one thread per instance on the (m+1) x m Hessenberg
//   V_{j+1} = w / h, Z_{j+1} = t / h
// Vectors are cut into chunks of kChunk elements that never straddle two instances; every
// dot product is a sum of per-chunk partials taken in chunk order, so an instance's result
// does not depend on what else is in the batch.  The host drives the cycles and reads one
// counter of still-running instances every kCheck steps (a stream synchronisation).
// Arithmetic is float64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sgn_2d.h"
#include "sgn_internal.h"

namespace sgn {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;                    // vector elements per chunk
constexpr int kPer = kChunk / kThreads;         // elements per thread
constexpr int kCheck = 4;                       // Arnoldi steps between host checks

struct Chunk {
  int inst;
  int len;
  long long start;
};

// Per-instance GMRES state (device resident).
struct Gm {
  double bnorm;          // ||b||_2
  double beta;           // ||r||_2 at the start of the cycle (then the final true residual)
  double scale;          // 1 / (the norm the newest basis vector is divided by)
  int run;               // 1 while the instance's current cycle goes on
  int in_cycle;          // 1 if the instance took part in the current cycle
  int j;                 // Arnoldi steps of the current cycle
  int steps;             // Arnoldi steps in total
  int cycles;
  int status;
  int done;              // 1 once the instance has its final status
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];   // fixed order
  return s;                                                // valid in thread 0
}

// partial[c][k] = Z_k . w over chunk c for k = 0..j (= <w, V_k> in the A^{-1} inner product)
__global__ void __launch_bounds__(kThreads) k_gm_dots(const Chunk* __restrict__ chunks,
                                                      const Gm* __restrict__ gm,
                                                      const double* __restrict__ Z,
                                                      long long vlen, const double* __restrict__ w,
                                                      int j, int ld,
                                                      double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const Chunk c = chunks[blockIdx.x];
  if (!gm[c.inst].run) return;
  double wr[kPer];
#pragma unroll
  for (int e = 0; e < kPer; ++e) {
    const int i = e * kThreads + threadIdx.x;
    wr[e] = i < c.len ? w[c.start + i] : 0.0;
  }
  for (int k = 0; k <= j; ++k) {
    const double* v = Z + (long long)k * vlen + c.start;
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int i = e * kThreads + threadIdx.x;
      if (i < c.len) acc += wr[e] * v[i];
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * ld + k] = s;
  }
}

// partial[c][0] = p . q over chunk c, for the running instances (run_only) or for every
// instance not finished yet
__global__ void __launch_bounds__(kThreads) k_gm_dot2(const Chunk* __restrict__ chunks,
                                                      const Gm* __restrict__ gm,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q, int run_only,
                                                      int ld, double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const Chunk c = chunks[blockIdx.x];
  if (run_only ? !gm[c.inst].run : gm[c.inst].done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < c.len; i += kThreads) acc += p[c.start + i] * q[c.start + i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partial[(long long)blockIdx.x * ld] = s;
}

// h_k = sum over the instance's chunks of partial[.][k]; w -= sum_k h_k V_k and
// t -= sum_k h_k Z_k (t stays A^{-1} w); the instance's first chunk adds h into column j of
// its Hessenberg matrix.
__global__ void __launch_bounds__(kThreads) k_gm_orth(const Chunk* __restrict__ chunks,
                                                      const int* __restrict__ first,
                                                      const int* __restrict__ nchunk,
                                                      const Gm* __restrict__ gm,
                                                      const double* __restrict__ V,
                                                      const double* __restrict__ Z, long long vlen,
                                                      double* __restrict__ w,
                                                      double* __restrict__ t, int j, int ld,
                                                      const double* __restrict__ partial,
                                                      double* __restrict__ H, int m) {
  __shared__ double h[SGN_GMRES_MAX_RESTART + 1];
  const Chunk c = chunks[blockIdx.x];
  if (!gm[c.inst].run) return;
  const int c0 = first[c.inst], nc = nchunk[c.inst];
  for (int k = threadIdx.x; k <= j; k += kThreads) {
    double s = 0.0;
    for (int q = 0; q < nc; ++q) s += partial[(long long)(c0 + q) * ld + k];
    h[k] = s;
  }
  __syncthreads();
  if (blockIdx.x == c0)
    for (int k = threadIdx.x; k <= j; k += kThreads)
      H[(long long)c.inst * (m + 1) * m + (long long)k * m + j] += h[k];
  for (int i = threadIdx.x; i < c.len; i += kThreads) {
    const long long q = c.start + i;
    double aw = w[q], at = t[q];
    for (int k = 0; k <= j; ++k) {
      aw -= h[k] * V[(long long)k * vlen + q];
      at -= h[k] * Z[(long long)k * vlen + q];
    }
    w[q] = aw;
    t[q] = at;
  }
}

// One thread per instance: sqrt(w.t) into H[j+1][j], the earlier rotations and a new one on
// column j, the rotated right-hand side, and the stopping decisions.
__global__ void k_gm_givens(int count, const int* __restrict__ first,
                            const int* __restrict__ nchunk, Gm* __restrict__ gm,
                            const double* __restrict__ partial, int ld, double* __restrict__ H,
                            double* __restrict__ cs, double* __restrict__ sn,
                            double* __restrict__ g, int m, int j, double rtol, int maxit,
                            int* __restrict__ running) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  Gm& s = gm[i];
  if (!s.run) return;
  double nn = 0.0;
  for (int q = 0; q < nchunk[i]; ++q) nn += partial[(long long)(first[i] + q) * ld];
  const double hn = isfinite(nn) ? sqrt(fmax(nn, 0.0)) : nn;   // NaN reaches den below
  double* Hi = H + (long long)i * (m + 1) * m;
  double* ci = cs + (long long)i * m;
  double* si = sn + (long long)i * m;
  double* gi = g + (long long)i * (m + 1);
  Hi[(long long)(j + 1) * m + j] = hn;
  for (int k = 0; k < j; ++k) {
    const double a = Hi[(long long)k * m + j], b = Hi[(long long)(k + 1) * m + j];
    Hi[(long long)k * m + j] = ci[k] * a + si[k] * b;
    Hi[(long long)(k + 1) * m + j] = -si[k] * a + ci[k] * b;
  }
  const double a = Hi[(long long)j * m + j];
  const double den = hypot(a, hn);
  s.j = j + 1;
  s.steps += 1;
  if (!(den > 0.0) || !isfinite(den)) {          // NaN / Inf, or a zero column
    s.status = SGN_ERR_BREAKDOWN;
    s.run = 0;
    s.done = 1;
    s.j = j;                                     // the column is unusable
    return;
  }
  ci[j] = a / den;
  si[j] = hn / den;
  Hi[(long long)j * m + j] = den;
  Hi[(long long)(j + 1) * m + j] = 0.0;
  gi[j + 1] = -si[j] * gi[j];
  gi[j] = ci[j] * gi[j];
  s.scale = hn > 0.0 ? 1.0 / hn : 0.0;
  if (fabs(gi[j + 1]) <= rtol * s.bnorm || hn == 0.0 || j + 1 == m || s.steps >= maxit)
    s.run = 0;
  else
    atomicAdd(running, 1);
}

// V_{j+1} = w * scale, Z_{j+1} = t * scale for the instances still running
__global__ void __launch_bounds__(kThreads) k_gm_scale(const Chunk* __restrict__ chunks,
                                                       const Gm* __restrict__ gm,
                                                       const double* __restrict__ w,
                                                       const double* __restrict__ t,
                                                       double* __restrict__ vout,
                                                       double* __restrict__ zout) {
  const Chunk c = chunks[blockIdx.x];
  const Gm& s = gm[c.inst];
  if (!s.run) return;
  for (int i = threadIdx.x; i < c.len; i += kThreads) {
    vout[c.start + i] = w[c.start + i] * s.scale;
    zout[c.start + i] = t[c.start + i] * s.scale;
  }
}

// End of a cycle: y from the triangular system (one thread per instance)
__global__ void k_gm_solve_y(int count, const Gm* __restrict__ gm, const double* __restrict__ H,
                             const double* __restrict__ g, double* __restrict__ y, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || !gm[i].in_cycle) return;
  const int k = gm[i].j;
  const double* Hi = H + (long long)i * (m + 1) * m;
  const double* gi = g + (long long)i * (m + 1);
  double* yi = y + (long long)i * m;
  for (int r = k - 1; r >= 0; --r) {
    double acc = gi[r];
    for (int q = r + 1; q < k; ++q) acc -= Hi[(long long)r * m + q] * yi[q];
    yi[r] = acc / Hi[(long long)r * m + r];
  }
}

// x += sum_k y_k Z_k over the instance's j basis vectors (Z = A^{-1} V), for the instances
// of the cycle
__global__ void __launch_bounds__(kThreads) k_gm_update_x(const Chunk* __restrict__ chunks,
                                                          const Gm* __restrict__ gm,
                                                          const double* __restrict__ Z,
                                                          long long vlen,
                                                          const double* __restrict__ y, int m,
                                                          double* __restrict__ x) {
  const Chunk c = chunks[blockIdx.x];
  const Gm& s = gm[c.inst];
  if (!s.in_cycle) return;
  const int k = s.j;
  const double* yi = y + (long long)c.inst * m;
  for (int i = threadIdx.x; i < c.len; i += kThreads) {
    const long long q = c.start + i;
    double acc = x[q];
    for (int t = 0; t < k; ++t) acc += yi[t] * Z[(long long)t * vlen + q];
    x[q] = acc;
  }
}

// r = b - Gx for the instances not finished
__global__ void __launch_bounds__(kThreads) k_gm_sub(const Chunk* __restrict__ chunks,
                                                     const Gm* __restrict__ gm,
                                                     const double* __restrict__ b,
                                                     const double* __restrict__ Gx,
                                                     double* __restrict__ r) {
  const Chunk c = chunks[blockIdx.x];
  if (gm[c.inst].done) return;
  for (int i = threadIdx.x; i < c.len; i += kThreads)
    r[c.start + i] = b[c.start + i] - Gx[c.start + i];
}

// mode 1 (start): sqrt(b.A^{-1}b); zero-rhs and bad-coefficient instances finish at once.
// mode 0 (restart): the true residual measure sqrt(r.A^{-1}r); finish, or start a cycle.
__global__ void k_gm_restart(int count, const int* __restrict__ first,
                             const int* __restrict__ nchunk, Gm* __restrict__ gm,
                             const SolveRec* __restrict__ coef, const double* __restrict__ partial,
                             int ld, double* __restrict__ H, double* __restrict__ g, int m,
                             double rtol, int maxit, int mode, int* __restrict__ running) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  Gm& s = gm[i];
  double nn = 0.0;
  for (int q = 0; q < nchunk[i]; ++q) nn += partial[(long long)(first[i] + q) * ld];
  const double nrm = sqrt(fmax(nn, 0.0));
  if (mode == 1) {
    const bool bad = !isfinite(nn);               // fmax(NaN, 0) is 0: test the sum itself
    s = Gm{};
    s.bnorm = nrm;
    if (coef[i].status != SGN_OK) {
      s.status = coef[i].status;
      s.done = 1;
    } else if (bad) {
      s.status = SGN_ERR_BREAKDOWN;
      s.done = 1;
    } else if (nrm == 0.0) {
      s.status = SGN_OK;                          // x = 0 (set by the caller's launch)
      s.done = 1;
    }
    return;
  }
  s.run = 0;
  s.in_cycle = 0;
  if (s.done) return;
  s.beta = nrm;
  if (!isfinite(nn)) {
    s.status = SGN_ERR_BREAKDOWN;
    s.done = 1;
  } else if (nrm <= rtol * s.bnorm) {
    s.status = SGN_OK;
    s.done = 1;
  } else if (s.steps >= maxit) {
    s.status = SGN_ERR_NOT_CONVERGED;
    s.done = 1;
  } else {
    s.run = 1;
    s.in_cycle = 1;
    s.j = 0;
    s.cycles += 1;
    s.scale = 1.0 / nrm;
    double* Hi = H + (long long)i * (m + 1) * m;
    for (int k = 0; k < (m + 1) * m; ++k) Hi[k] = 0.0;
    double* gi = g + (long long)i * (m + 1);
    for (int k = 0; k <= m; ++k) gi[k] = 0.0;
    gi[0] = nrm;
    atomicAdd(running, 1);
  }
}

// x = 0 for the instances with b = 0
__global__ void __launch_bounds__(kThreads) k_gm_zero_x(const Chunk* __restrict__ chunks,
                                                        const Gm* __restrict__ gm,
                                                        double* __restrict__ x) {
  const Chunk c = chunks[blockIdx.x];
  const Gm& s = gm[c.inst];
  if (!(s.done && s.status == SGN_OK && s.bnorm == 0.0)) return;
  for (int i = threadIdx.x; i < c.len; i += kThreads) x[c.start + i] = 0.0;
}

// Reports into the solve records: iters = steps, refinements = cycles, ratio = the true
// sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b), status.
__global__ void k_gm_report(int count, const Gm* __restrict__ gm, SolveRec* __restrict__ rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const Gm& s = gm[i];
  rec[i].iters = s.steps;
  rec[i].refinements = s.cycles;
  rec[i].ratio = s.bnorm > 0.0 ? s.beta / s.bnorm : 0.0;
  rec[i].status = s.done ? s.status : SGN_ERR_NOT_CONVERGED;
}

}  // namespace

cudaError_t run_gmres(const GmresArgs& a, cudaStream_t s) {
  const int m = a.restart, count = a.count;
  // chunk table: chunks never straddle instances; in 2d the one instance owns both planes
  std::vector<Chunk> ch;
  std::vector<int> first(count), nch(count);
  for (int i = 0; i < count; ++i) {
    const long long b0 = a.dim == 1 ? a.offsets[i] : 0;
    const long long len = a.dim == 1 ? a.offsets[i + 1] - a.offsets[i] : a.vec_len;
    first[i] = (int)ch.size();
    for (long long o = 0; o < len; o += kChunk)
      ch.push_back(Chunk{i, (int)std::min<long long>(kChunk, len - o), b0 + o});
    nch[i] = (int)ch.size() - first[i];
  }
  const int nc = (int)ch.size();
  const int ld = m + 1;
  const long long vlen = a.vec_len;
  const size_t vbytes = sizeof(double) * (size_t)vlen;
  // workspace: bases V and Z (m+1 vectors each), w, t; chunk tables; partials; per-instance
  // state, Hessenberg matrices, rotations, right-hand sides and solutions
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oV = take(vbytes * (m + 1)), oZ = take(vbytes * (m + 1)), oW = take(vbytes),
               oT = take(vbytes);
  const size_t oCh = take(sizeof(Chunk) * nc), oFi = take(sizeof(int) * count),
               oNc = take(sizeof(int) * count);
  const size_t oP = take(sizeof(double) * (size_t)nc * ld);
  const size_t oGm = take(sizeof(Gm) * count);
  const size_t oH = take(sizeof(double) * (size_t)count * (m + 1) * m);
  const size_t oCs = take(sizeof(double) * (size_t)count * m),
               oSn = take(sizeof(double) * (size_t)count * m),
               oG = take(sizeof(double) * (size_t)count * (m + 1)),
               oY = take(sizeof(double) * (size_t)count * m);
  const size_t oRun = take(sizeof(int));
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), off, s);
  if (e != cudaSuccess) return e;
  int* h_run = nullptr;
  e = cudaMallocHost(reinterpret_cast<void**>(&h_run), sizeof(int));
  if (e != cudaSuccess) {
    cudaFreeAsync(base, s);
    return e;
  }
  double* V = reinterpret_cast<double*>(base + oV);
  double* Z = reinterpret_cast<double*>(base + oZ);
  double* w = reinterpret_cast<double*>(base + oW);
  double* t = reinterpret_cast<double*>(base + oT);
  Chunk* d_ch = reinterpret_cast<Chunk*>(base + oCh);
  int* d_fi = reinterpret_cast<int*>(base + oFi);
  int* d_nc = reinterpret_cast<int*>(base + oNc);
  double* partial = reinterpret_cast<double*>(base + oP);
  Gm* gm = reinterpret_cast<Gm*>(base + oGm);
  double* H = reinterpret_cast<double*>(base + oH);
  double* cs = reinterpret_cast<double*>(base + oCs);
  double* sn = reinterpret_cast<double*>(base + oSn);
  double* g = reinterpret_cast<double*>(base + oG);
  double* y = reinterpret_cast<double*>(base + oY);
  int* run = reinterpret_cast<int*>(base + oRun);
  const int ib = (count + 127) / 128;

  auto precond = [&](const double* r, double* out) {
    return a.dim == 1 ? launch_precond1d(*a.l1, a.tw64, a.coef, r, out, s)
                      : launch_precond2d(*a.l2, a.tw64, a.coef, r, out, s);
  };
  auto applyG = [&](const double* u, double* out) {
    return a.dim == 1 ? launch_apply_G1d(*a.l1, a.tw64, a.eta, a.gradh, u, out, s)
                      : launch_apply_G2d(*a.l2, a.tw64, a.eta, a.gradh, u, out, s);
  };
  auto read_running = [&](int& n) -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(h_run, run, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (r == cudaSuccess) r = cudaStreamSynchronize(s);
    n = *h_run;
    return r;
  };
#define GM_TRY(x)                   \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) goto out; \
  } while (0)
  {
    int nrun = 0;
    GM_TRY(cudaMemcpyAsync(d_ch, ch.data(), sizeof(Chunk) * nc, cudaMemcpyHostToDevice, s));
    GM_TRY(cudaMemcpyAsync(d_fi, first.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    GM_TRY(cudaMemcpyAsync(d_nc, nch.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    GM_TRY(cudaMemsetAsync(base + oV, 0, oCh - oV, s));          // V, Z, w, t
    GM_TRY(cudaMemsetAsync(gm, 0, sizeof(Gm) * count, s));
    // sqrt(b.A^{-1}b) per instance
    GM_TRY(precond(a.b, t));
    k_gm_dot2<<<nc, kThreads, 0, s>>>(d_ch, gm, a.b, t, 0, ld, partial);
    GM_TRY(cudaGetLastError());
    k_gm_restart<<<ib, 128, 0, s>>>(count, d_fi, d_nc, gm, a.coef, partial, ld, H, g, m, a.rtol,
                                    a.maxit, 1, run);
    GM_TRY(cudaGetLastError());
    k_gm_zero_x<<<nc, kThreads, 0, s>>>(d_ch, gm, a.x);
    GM_TRY(cudaGetLastError());
    for (;;) {
      // true residual r = b - G x into V_0, A^{-1} r into Z_0, then finish or start a cycle
      GM_TRY(applyG(a.x, w));
      k_gm_sub<<<nc, kThreads, 0, s>>>(d_ch, gm, a.b, w, V);
      GM_TRY(cudaGetLastError());
      GM_TRY(precond(V, Z));
      k_gm_dot2<<<nc, kThreads, 0, s>>>(d_ch, gm, V, Z, 0, ld, partial);
      GM_TRY(cudaGetLastError());
      GM_TRY(cudaMemsetAsync(run, 0, sizeof(int), s));
      k_gm_restart<<<ib, 128, 0, s>>>(count, d_fi, d_nc, gm, a.coef, partial, ld, H, g, m,
                                      a.rtol, a.maxit, 0, run);
      GM_TRY(cudaGetLastError());
      GM_TRY(read_running(nrun));
      if (nrun == 0) break;
      k_gm_scale<<<nc, kThreads, 0, s>>>(d_ch, gm, V, Z, V, Z);      // divide by the norm
      GM_TRY(cudaGetLastError());
      for (int j = 0; j < m; ++j) {
        GM_TRY(applyG(Z + (long long)j * vlen, w));
        GM_TRY(precond(w, t));
        for (int pass = 0; pass < 2; ++pass) {
          k_gm_dots<<<nc, kThreads, 0, s>>>(d_ch, gm, Z, vlen, w, j, ld, partial);
          GM_TRY(cudaGetLastError());
          k_gm_orth<<<nc, kThreads, 0, s>>>(d_ch, d_fi, d_nc, gm, V, Z, vlen, w, t, j, ld,
                                            partial, H, m);
          GM_TRY(cudaGetLastError());
        }
        k_gm_dot2<<<nc, kThreads, 0, s>>>(d_ch, gm, w, t, 1, ld, partial);
        GM_TRY(cudaGetLastError());
        GM_TRY(cudaMemsetAsync(run, 0, sizeof(int), s));
        k_gm_givens<<<ib, 128, 0, s>>>(count, d_fi, d_nc, gm, partial, ld, H, cs, sn, g, m, j,
                                       a.rtol, a.maxit, run);
        GM_TRY(cudaGetLastError());
        // the host looks at the running count every kCheck steps (and at the cycle's end):
        // instances that stopped skip the steps launched in between
        if ((j + 1) % kCheck == 0 || j + 1 == m) {
          GM_TRY(read_running(nrun));
          if (nrun == 0) break;
        }
        k_gm_scale<<<nc, kThreads, 0, s>>>(d_ch, gm, w, t, V + (long long)(j + 1) * vlen,
                                           Z + (long long)(j + 1) * vlen);
        GM_TRY(cudaGetLastError());
      }
      // x += Z y for the instances of this cycle
      k_gm_solve_y<<<ib, 128, 0, s>>>(count, gm, H, g, y, m);
      GM_TRY(cudaGetLastError());
      k_gm_update_x<<<nc, kThreads, 0, s>>>(d_ch, gm, Z, vlen, y, m, a.x);
      GM_TRY(cudaGetLastError());
    }
    k_gm_report<<<ib, 128, 0, s>>>(count, gm, a.rec);
    GM_TRY(cudaGetLastError());
  }
#undef GM_TRY
out:
  cudaError_t e2 = cudaFreeAsync(base, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  cudaFreeHost(h_run);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  return e;
}

}  // namespace sgn
