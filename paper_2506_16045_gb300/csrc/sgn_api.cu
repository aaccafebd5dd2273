// C ABI of the SGN library: contexts, batch layouts, the hot-path entry points and the
// time integrators (host orchestration of the kernels in sgn_1d.cu / sgn_2d.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <utility>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sgn.h"
#include "sgn_internal.h"
#include "sgn_2d.h"

using sgn::Inst1d;
using sgn::Layout1d;
using sgn::SolveRec;

struct ProfRec {
  cudaEvent_t a, b;
  int kind;              // 0 = PCG launch group, 1 = right-hand side launch group
};

// A profiled launch group inside a captured graph: its two event-record nodes, which get
// fresh events before every replay (so replays accumulate without synchronising).
struct CapRec {
  cudaGraphNode_t a, b;
  int kind;
};

struct sgn_ctx {
  int device = 0;
  void* tw64 = nullptr;
  void* tw32 = nullptr;
  std::string err;
  int prof = 0;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  std::vector<CapRec>* capture = nullptr;   // non-null while a profiled step is captured
};

namespace {
// Brackets one launch group with events when profiling is on.
struct ProfScope {
  sgn_ctx* ctx;
  cudaStream_t s;
  ProfRec r{};
  bool on;
  cudaGraphNode_t na = nullptr;
  ProfScope(sgn_ctx* c, cudaStream_t st, int kind) : ctx(c), s(st), on(c && c->prof) {
    if (!on) return;
    r.kind = kind;
    r.a = take();
    r.b = take();
    if (ctx->capture) {
      na = record_node(r.a);
    } else {
      cudaEventRecord(r.a, s);
    }
  }
  // during capture: an external event-record node (it records a timestamp on replay); the
  // stream's dependency set right after the record is that node
  cudaGraphNode_t record_node(cudaEvent_t e) {
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess ||
        nd != 1)
      return nullptr;
    return deps[0];
  }
  cudaEvent_t take() {
    cudaEvent_t e;
    if (!ctx->pool.empty()) {
      e = ctx->pool.back();
      ctx->pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  ~ProfScope() {
    if (!on) return;
    if (ctx->capture) {
      const cudaGraphNode_t nb = record_node(r.b);
      if (na && nb) ctx->capture->push_back(CapRec{na, nb, r.kind});
      ctx->pool.push_back(r.a);   // the replays use their own events
      ctx->pool.push_back(r.b);
      return;
    }
    cudaEventRecord(r.b, s);
    ctx->recs.push_back(r);
  }
};
}  // namespace

struct sgn_layout {
  sgn_ctx* ctx = nullptr;
  int device = 0;                   // copied from ctx: destroying a layout never reads ctx
  int count = 0;
  int dim = 1;
  std::vector<sgn_grid> grids;
  std::vector<long long> offsets;
  long long points = 0;
  Layout1d l1;
  sgn::Layout2d l2;
  sgn::Batch2d b2;                  // 2d layouts of count > 1: instances 1.. and batch buffers
  void* ws = nullptr;               // spectral workspace
  double* scratch = nullptr;        // 5 P doubles (rhs intermediates)
  float* coef_df = nullptr;         // 6 P floats (double-float coefficients, high and low parts)
  SolveRec* rec = nullptr;          // [count] per-instance solve reports
  SolveRec* given = nullptr;        // [count] caller-provided coefficients
};

namespace {

struct DevStats {
  long long solves;
  long long iterations;
  int max_iters;
  int status;
  double flops32;        // algorithmic float32 flops of the PCG solves
  double flops64;        // algorithmic float64 flops of the PCG solves
  long long refinements; // float32 inner solves (mixed)
  long long sbdf2_warn;  // SBDF2 instance-steps whose eta_max left the fixed A's stable range
  unsigned long long guard_max;   // 2d guard: running eta_max (order-preserving bits)
  unsigned int guard_ticket;      // 2d guard: blocks done
};

// Order-preserving unsigned image of a double (for atomicMax over doubles of any sign).
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long o) {
  return __longlong_as_double((long long)((o >> 63) ? (o & 0x7fffffffffffffffull) : ~o));
}

// The SBDF2 guard of a 2d state (reading R10, below) over many blocks: each block's eta_max
// goes to one atomicMax; the last block to finish compares it with the fixed A's eta_max,
// counts a warning, and resets the running maximum for the next step.
__global__ void __launch_bounds__(256) k_sbdf2_guard2d(long long P, const double* __restrict__ eta,
                                                       const SolveRec* __restrict__ A,
                                                       DevStats* __restrict__ stats) {
  __shared__ double red[8];
  __shared__ bool last;
  double m = -1e300;
  for (long long j = blockIdx.x * 256ll + threadIdx.x; j < P; j += (long long)gridDim.x * 256)
    m = fmax(m, eta[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    m = fmax(m, red[0]);
    atomicMax(&stats->guard_max, ordered_bits(m));
    __threadfence();
    last = atomicAdd(&stats->guard_ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  const double mx = from_ordered(atomicExch(&stats->guard_max, 0ull));
  stats->guard_ticket = 0;
  const double r = mx / A->eta_max;
  if (!(r * r * r < 4.0 / 3.0)) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->sbdf2_warn), 1ull);
}

// SBDF2 guard (reading R10): A is fixed from the initial data; the generalised eigenvalues
// of A^{-1} G grow like (eta_max / eta_max,0)^3, and SBDF2's zero-stability needs them below
// 4/3.  One block per instance takes the level's eta_max and counts the instances past
// that ratio.  (1d: insts; 2d: one instance of P points.)
__global__ void k_sbdf2_guard(const Inst1d* __restrict__ insts, long long P,
                              const double* __restrict__ eta, const SolveRec* __restrict__ A,
                              DevStats* __restrict__ stats) {
  __shared__ double red[32];
  const long long off = insts ? insts[blockIdx.x].off : 0;
  const long long n = insts ? insts[blockIdx.x].n : P;
  double m = -1e300;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, eta[off + j]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    m = fmax(m, red[0]);
    const double r = m / A[blockIdx.x].eta_max;
    if (!(r * r * r < 4.0 / 3.0)) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->sbdf2_warn), 1ull);
  }
}

// Algorithmic flop model of one solve on n points (complex FFT of length n: 5 n log2 n):
//   inner iteration: 2 FFTs + pointwise/vector work = 10 n log2 n + 26 n
//   float64 residual pass: 10 n log2 n + 20 n; transforms of b, x0 and the result: 5 n log2 n
__device__ void solve_flops(double n, double lg, int iters, int refinements, int mixed,
                            double& f32, double& f64) {
  const double it = 10.0 * n * lg + 26.0 * n;
  const double res = 10.0 * n * lg + 20.0 * n;
  if (mixed) {
    f32 = iters * it;
    f64 = 5.0 * n * lg + (refinements + 1) * res;
  } else {
    f32 = 0.0;
    f64 = 10.0 * n * lg + res + iters * it;
  }
}

// One thread per instance; the counters are summed with atomics (one block).
__global__ void k_accum(const SolveRec* __restrict__ rec, const Inst1d* __restrict__ insts,
                        int count, long long n2d, int log2n2d, int mixed, DevStats* st) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->solves), 1ull);
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->iterations),
              (unsigned long long)rec[i].iters);
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->refinements),
              (unsigned long long)rec[i].refinements);
    atomicMax(&st->max_iters, rec[i].iters);
    atomicMax(&st->status, rec[i].status);
    double f32, f64;
    const double n = insts ? (double)insts[i].n : (double)n2d;
    // log2 n (the generic sizes, log2n = 0: the real logarithm)
    const double lg = insts ? (insts[i].log2n ? (double)insts[i].log2n : log2((double)insts[i].n))
                            : (double)log2n2d;
    solve_flops(n, lg, rec[i].iters, rec[i].refinements, mixed, f32, f64);
    atomicAdd(&st->flops32, f32);
    atomicAdd(&st->flops64, f64);
  }
}

// out = sum_t a_t x_t + dt_i sum_t c_t f_t over the points of each instance
struct LinComb {
  const double* x[4];
  double a[4];
  int nx;
  const double* f[4];
  double c[4];
  int nf;
};

// Up to two combinations in one launch (blockIdx.z selects), each over all instances
// (blockIdx.y) in chunks of kLinChunk points (blockIdx.x), so large instances do not
// serialise the launch.
struct LinJob {
  double* out;
  LinComb lc;
  int components;
};
struct LinJobs {
  LinJob j[2];
};
constexpr int kLinChunk = 1024;

__global__ void __launch_bounds__(256) k_lincomb(const Inst1d* __restrict__ insts,
                                                 const double* __restrict__ dt,
                                                 const __grid_constant__ LinJobs J,
                                                 long long plane) {
  const LinJob& jb = J.j[blockIdx.z];
  const Inst1d I = insts[blockIdx.y];
  const int j0 = blockIdx.x * kLinChunk;
  if (j0 >= I.n) return;
  const int j1 = min(I.n, j0 + kLinChunk);
  const double d = dt[blockIdx.y];
  for (int comp = 0; comp < jb.components; ++comp) {
    for (int j = j0 + threadIdx.x; j < j1; j += 256) {
      const long long q = comp * plane + I.off + j;
      double acc = 0.0, accf = 0.0;
      for (int t = 0; t < jb.lc.nx; ++t) acc += jb.lc.a[t] * jb.lc.x[t][q];
      for (int t = 0; t < jb.lc.nf; ++t) accf += jb.lc.c[t] * jb.lc.f[t][q];
      jb.out[q] = acc + d * accf;
    }
  }
}

// External forcing of the steppers (Test 1 of §6.4, manufactured solutions): a finite
// Fourier series in time, f_eta += sum_k cos(omega_k tau + theta_k) phi_eta_k and likewise
// for f_U, at the stage time tau = t_i + c dt_i of every instance.
struct ForceTerms {
  const double* pe[SGN_MAX_FORCING];    // phi_eta_k, packed like eta (P doubles)
  const double* pu[SGN_MAX_FORCING];    // phi_U_k, packed like U (d P doubles)
  double omega[SGN_MAX_FORCING];
  double theta[SGN_MAX_FORCING];
  int K;
};

// insts == nullptr: one instance of n2d points (a 2d layout)
__global__ void __launch_bounds__(256) k_force(const Inst1d* __restrict__ insts,
                                               const double* __restrict__ tnow,
                                               const double* __restrict__ dt, double c,
                                               const __grid_constant__ ForceTerms F,
                                               double* __restrict__ fe, double* __restrict__ fU,
                                               long long plane, int d, long long n2d) {
  __shared__ double w[SGN_MAX_FORCING];
  const int i = blockIdx.y;
  const long long off = insts ? insts[i].off : 0;
  const long long n = insts ? insts[i].n : n2d;
  const long long j0 = (long long)blockIdx.x * kLinChunk;
  if (j0 >= n) return;                                  // uniform over the block
  if (threadIdx.x < F.K) {
    const double tau = tnow[i] + c * dt[i];
    w[threadIdx.x] = cos(F.omega[threadIdx.x] * tau + F.theta[threadIdx.x]);
  }
  __syncthreads();
  const long long j1 = j0 + kLinChunk < n ? j0 + kLinChunk : n;
  for (long long j = j0 + threadIdx.x; j < j1; j += 256) {
    const long long q = off + j;
    double ae = 0.0;
    for (int k = 0; k < F.K; ++k) ae += w[k] * F.pe[k][q];
    fe[q] += ae;
    for (int comp = 0; comp < d; ++comp) {
      const long long qc = comp * plane + q;
      double au = 0.0;
      for (int k = 0; k < F.K; ++k) au += w[k] * F.pu[k][qc];
      fU[qc] += au;
    }
  }
}

// t_i += dt_i: per-instance simulated time on the device (read by k_force; advanced inside
// captured steps, so a replayed graph keeps it current)
__global__ void k_advance_time(double* __restrict__ t, const double* __restrict__ dt, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) t[i] += dt[i];
}

sgn_status fail(sgn_ctx* ctx, sgn_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

sgn_status cuda_fail(sgn_ctx* ctx, cudaError_t e, const char* where) {
  cudaGetLastError();   // a failed call also sets the runtime's last error: do not pass it on
  if (e == cudaErrorMemoryAllocation)
    return fail(ctx, SGN_ERR_NOMEM, std::string(where) + ": out of device memory");
  return fail(ctx, SGN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SGN_CUDA(ctx, expr)                                   \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr); \
  } while (0)

inline cudaStream_t as_stream(sgn_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// a layout holding sizes that are not powers of two (the generic kernels)
bool has_generic(const sgn_layout* lay) {
  if (lay->dim == 2) return lay->l2.mr;
  return lay->l1.class_end[sgn::kGenericClass] > lay->l1.class_begin[sgn::kGenericClass];
}

int ilog2_exact(int n) {
  if (n <= 0 || (n & (n - 1))) return -1;
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

sgn_status check_layout(const sgn_layout* lay) {
  if (!lay || !lay->ctx) return SGN_ERR_INVALID_ARG;
  return SGN_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

// =======================================================================================
// Context
// =======================================================================================

extern "C" const char* sgn_status_string(sgn_status s) {
  switch (s) {
    case SGN_OK: return "ok";
    case SGN_ERR_INVALID_ARG: return "invalid argument";
    case SGN_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case SGN_ERR_NOMEM: return "out of device memory";
    case SGN_ERR_CUDA: return "CUDA error";
    case SGN_ERR_NOT_CONVERGED: return "not converged";
    case SGN_ERR_BREAKDOWN: return "PCG breakdown";
    case SGN_ERR_NONPOSITIVE_DEPTH: return "non-positive depth";
    case SGN_ERR_PENDING: return "pending";
    case SGN_ERR_TIMEOUT: return "timeout";
    case SGN_ERR_REJECTED: return "rejected";
  }
  return "unknown status";
}

extern "C" sgn_status sgn_create(sgn_ctx** out, int device, size_t workspace_bytes) {
  (void)workspace_bytes;
  if (!out) return SGN_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  sgn_ctx* ctx = new (std::nothrow) sgn_ctx();
  if (!ctx) return SGN_ERR_NOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  if (cudaMalloc(&ctx->tw64, sizeof(double) * 2 * sgn::kTwiddleN) != cudaSuccess ||
      cudaMalloc(&ctx->tw32, sgn::kTw32Bytes + sgn::kTwDfBytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->tw64);
    delete ctx;
    return SGN_ERR_NOMEM;
  }
  if (sgn::twiddles_init(ctx->tw64, ctx->tw32, 0) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->tw64);
    cudaFree(ctx->tw32);
    delete ctx;
    return SGN_ERR_CUDA;
  }
  *out = ctx;
  return SGN_OK;
}

extern "C" sgn_status sgn_profile_enable(sgn_ctx* ctx, int on) {
  if (!ctx) return SGN_ERR_INVALID_ARG;
  ctx->prof = on ? 1 : 0;
  return SGN_OK;
}

extern "C" sgn_status sgn_profile_inner2d(sgn_layout* lay, int on, double* ms,
                                          long long* launches, long long* iterations) {
  if (check_layout(lay) || lay->dim != 2) return SGN_ERR_INVALID_ARG;
  if (lay->l2.mr) return SGN_ERR_UNSUPPORTED_SIZE;    // no persistent inner solve
  DeviceGuard g(lay->device);
  sgn::Layout2d& L = lay->l2;
  double t = 0.0;
  long long n = 0, it = 0;
  if (L.prof) {
    for (size_t i = 0; i < L.prof->a.size(); ++i) {
      float f = 0.0f;
      if (cudaEventSynchronize(L.prof->b[i]) != cudaSuccess ||
          cudaEventElapsedTime(&f, L.prof->a[i], L.prof->b[i]) != cudaSuccess) {
        cudaGetLastError();
        return fail(lay->ctx, SGN_ERR_CUDA, "profile event");
      }
      t += f;
      n += 1;
      it += L.prof->iters[i];
      cudaEventDestroy(L.prof->a[i]);
      cudaEventDestroy(L.prof->b[i]);
    }
    delete L.prof;
    L.prof = nullptr;
  }
  if (on) L.prof = new (std::nothrow) sgn::Prof2d();
  if (on && !L.prof) return fail(lay->ctx, SGN_ERR_NOMEM, "profile record");
  if (ms) *ms = t;
  if (launches) *launches = n;
  if (iterations) *iterations = it;
  return SGN_OK;
}

extern "C" sgn_status sgn_profile_read(sgn_ctx* ctx, double* pcg_ms, long long* pcg_calls,
                                       double* rhs_ms, long long* rhs_calls) {
  if (!ctx) return SGN_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  double ms[2] = {0.0, 0.0};
  long long cnt[2] = {0, 0};
  for (ProfRec& r : ctx->recs) {
    float t = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SGN_ERR_CUDA, "profile event");
    }
    ms[r.kind] += t;
    cnt[r.kind] += 1;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  if (pcg_ms) *pcg_ms = ms[0];
  if (pcg_calls) *pcg_calls = cnt[0];
  if (rhs_ms) *rhs_ms = ms[1];
  if (rhs_calls) *rhs_calls = cnt[1];
  return SGN_OK;
}

extern "C" void sgn_destroy(sgn_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  for (ProfRec& r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  cudaFree(ctx->tw64);
  cudaFree(ctx->tw32);
  delete ctx;
}

extern "C" const char* sgn_last_error(const sgn_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

// =======================================================================================
// Layouts
// =======================================================================================

extern "C" sgn_status sgn_layout_create(sgn_ctx* ctx, int count, const sgn_grid* grids,
                                        sgn_layout** out) {
  if (!ctx || !grids || !out || count <= 0) return fail(ctx, SGN_ERR_INVALID_ARG, "layout args");
  *out = nullptr;
  const int dim = grids[0].dim;
  if (dim != 1 && dim != 2) return fail(ctx, SGN_ERR_INVALID_ARG, "dim must be 1 or 2");
  if (dim == 2 && count > sgn::kMaxBatch2dAbi)
    return fail(ctx, SGN_ERR_INVALID_ARG, "too many 2d instances in one layout");
  for (int i = 1; dim == 2 && i < count; ++i)
    if (grids[i].nx != grids[0].nx || grids[i].ny != grids[0].ny || grids[i].Lx != grids[0].Lx ||
        grids[i].Ly != grids[0].Ly || grids[i].g != grids[0].g)
      return fail(ctx, SGN_ERR_INVALID_ARG, "a 2d batch needs one grid for every instance");
  for (int i = 0; i < count; ++i) {
    const sgn_grid& g = grids[i];
    if (g.dim != dim || !(g.Lx > 0.0) || (dim == 2 && !(g.Ly > 0.0)))
      return fail(ctx, SGN_ERR_INVALID_ARG, "grid fields");
    if (dim == 1 && g.ny != 1) return fail(ctx, SGN_ERR_INVALID_ARG, "1d grid needs ny = 1");
    const int lx = ilog2_exact(g.nx);
    if (dim == 1 && (lx < 3 || lx > sgn::kMaxLog1d) && !(lx < 0 && sgn::mr_size_ok(g.nx)))
      return fail(ctx, SGN_ERR_UNSUPPORTED_SIZE,
                  "1d nx must be a power of two in [8, 16384] or 2^a 3^b 5^c (a >= 1) in [6, 16384]");
    if (dim == 2) {
      const int ly = ilog2_exact(g.ny);
      auto side = [](int n, int l) { return (l >= 3 && l <= 10) || sgn::mr2d_side_ok(n); };
      if (!side(g.nx, lx) || !side(g.ny, ly))
        return fail(ctx, SGN_ERR_UNSUPPORTED_SIZE,
                    "2d nx, ny must be powers of two in [8, 1024] or 2^a 3^b 5^c (a >= 1) "
                    "in [6, 1024]");
      if (count > 1 && (lx < 0 || ly < 0))
        return fail(ctx, SGN_ERR_UNSUPPORTED_SIZE, "2d batches take power-of-two grids");
    }
  }
  sgn_layout* lay = new (std::nothrow) sgn_layout();
  if (!lay) return SGN_ERR_NOMEM;
  lay->ctx = ctx;
  lay->device = ctx->device;
  lay->count = count;
  lay->dim = dim;
  lay->grids.assign(grids, grids + count);
  lay->offsets.resize(count + 1);
  long long off = 0;
  for (int i = 0; i < count; ++i) {
    lay->offsets[i] = off;
    off += (long long)grids[i].nx * grids[i].ny;
  }
  lay->offsets[count] = off;
  lay->points = off;
  DeviceGuard gd(ctx->device);
  auto cleanup = [&](sgn_status s, const char* msg) {
    sgn_layout_destroy(lay);
    return fail(ctx, s, msg);
  };
  if (dim == 1) {
    Layout1d& L = lay->l1;
    L.count = count;
    L.points = off;
    L.h_inst = new Inst1d[count];
    long long ws = 0;
    std::vector<int> ids;
    for (int l = 3; l <= sgn::kMaxLog1d; ++l) {
      L.class_begin[l] = (int)ids.size();
      for (int i = 0; i < count; ++i)
        if (ilog2_exact(grids[i].nx) == l) ids.push_back(i);
      L.class_end[l] = (int)ids.size();
    }
    L.class_begin[sgn::kGenericClass] = (int)ids.size();
    for (int i = 0; i < count; ++i)
      if (ilog2_exact(grids[i].nx) < 0) ids.push_back(i);
    L.class_end[sgn::kGenericClass] = (int)ids.size();
    std::vector<std::pair<int, long long>> tables;   // generic n and its twiddles' offset
    long long gbuf = 0;                              // global transform buffers (complex)
    for (int i = 0; i < count; ++i) {
      Inst1d& I = L.h_inst[i];
      I.n = grids[i].nx;
      I.log2n = ilog2_exact(I.n) < 0 ? 0 : ilog2_exact(I.n);
      I.L = grids[i].Lx;
      I.off = lay->offsets[i];
      I.ws = ws;
      I.tw = 0;
      I.gbuf = -1;
      ws += (long long)sgn::kWsVectors * (I.n / 2 + 1);
      L.maxn = std::max(L.maxn, I.n);
      if (I.log2n == 0) {
        auto it = std::find_if(tables.begin(), tables.end(),
                               [&](const std::pair<int, long long>& t) { return t.first == I.n; });
        if (it == tables.end()) {
          tables.emplace_back(I.n, L.mr_tw_len);
          I.tw = L.mr_tw_len;
          L.mr_tw_len += sgn::mr_twiddle_len(I.n);
        } else {
          I.tw = it->second;
        }
        if (sgn::mr_in_smem(I.n)) {
          L.mr_smem_n = std::max(L.mr_smem_n, I.n);
        } else {
          I.gbuf = gbuf;
          gbuf += 2LL * I.n;
        }
      }
    }
    L.mr_tw_len += L.mr_tw_len & 1;                 // the double-float table 16-byte aligned
    L.ws_cplx = ws;
    if (!tables.empty()) {
      // float64, float32 and double-float complex entries: 16 + 8 + 16 bytes each
      if (cudaMalloc(&L.mr_tw, (size_t)40 * L.mr_tw_len) != cudaSuccess ||
          (gbuf > 0 && cudaMalloc(&L.mr_big, (size_t)16 * gbuf) != cudaSuccess)) {
        cudaGetLastError();
        return cleanup(SGN_ERR_NOMEM, "layout allocation");
      }
      for (const auto& t : tables)
        if (sgn::mr_twiddles_init(t.first, t.second, L, nullptr) != cudaSuccess)
          return cleanup(SGN_ERR_CUDA, "twiddle tables");
      if (cudaStreamSynchronize(nullptr) != cudaSuccess)
        return cleanup(SGN_ERR_CUDA, "twiddle tables");
    }
    const int nbig = L.class_end[sgn::kMaxLog1d] - L.class_begin[sgn::kMaxLog1d];
    if (nbig > 0 &&
        cudaMalloc(&L.big, sizeof(double) * 2 * ((size_t)nbig << sgn::kMaxLog1d)) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(SGN_ERR_NOMEM, "layout allocation");
    }
    if (cudaMalloc(&L.d_inst, sizeof(Inst1d) * count) != cudaSuccess ||
        cudaMalloc(&L.d_ids, sizeof(int) * count) != cudaSuccess ||
        cudaMalloc(&lay->ws, sizeof(double) * 2 * ws) != cudaSuccess ||
        cudaMalloc(&lay->scratch, sizeof(double) * 5 * off) != cudaSuccess ||
        cudaMalloc(&lay->coef_df, sizeof(float) * 6 * off) != cudaSuccess ||
        cudaMalloc(&lay->rec, sizeof(SolveRec) * count) != cudaSuccess ||
        cudaMalloc(&lay->given, sizeof(SolveRec) * count) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(SGN_ERR_NOMEM, "layout allocation");
    }
    if (cudaMemcpy(L.d_inst, L.h_inst, sizeof(Inst1d) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(L.d_ids, ids.data(), sizeof(int) * count, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      return cleanup(SGN_ERR_CUDA, "layout upload");
    }
    int ncls = 0;
    for (int i = 0; i < sgn::kNumClassSlots; ++i) {
      const int l = sgn::class_at(i);
      ncls += L.class_end[l] > L.class_begin[l];
    }
    if (ncls > 1) {
      if (cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(SGN_ERR_CUDA, "layout events");
      // Side stream c carries the c-th largest class.  A solve CTA of the largest classes
      // needs a whole SM (its registers or shared memory), so their blocks must not queue
      // behind small classes spread over the SMs: larger classes get higher priorities,
      // and the block scheduler dispatches their pending blocks first.
      int lo = 0, hi = 0;   // cudaDeviceGetStreamPriorityRange: hi is the greatest priority
      if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
        cudaGetLastError();
        lo = hi = 0;
      }
      for (int c = 0; c < ncls; ++c) {
        const int prio = hi + c < lo ? hi + c : lo;   // numerically lower = higher priority
        if (cudaStreamCreateWithPriority(&L.side[c], cudaStreamNonBlocking, prio) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.join[c], cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          return cleanup(SGN_ERR_CUDA, "layout streams");
        }
      }
    }
  } else {
    cudaError_t e = sgn::layout2d_create(lay->l2, grids[0]);
    if (e == cudaSuccess && count > 1) e = sgn::batch2d_create(lay->b2, lay->l2, grids[0], count);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cleanup(e == cudaErrorMemoryAllocation ? SGN_ERR_NOMEM : SGN_ERR_CUDA, "2d layout");
    }
    if (cudaMalloc(&lay->rec, sizeof(SolveRec) * count) != cudaSuccess ||
        cudaMalloc(&lay->given, sizeof(SolveRec) * count) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(SGN_ERR_NOMEM, "layout allocation");
    }
  }
  *out = lay;
  return SGN_OK;
}

extern "C" void sgn_layout_destroy(sgn_layout* lay) {
  if (!lay) return;
  DeviceGuard g(lay->device);
  for (int c = 0; c < 16; ++c) {
    if (lay->l1.side[c]) cudaStreamDestroy(lay->l1.side[c]);
    if (lay->l1.join[c]) cudaEventDestroy(lay->l1.join[c]);
  }
  if (lay->l1.fork) cudaEventDestroy(lay->l1.fork);
  cudaFree(lay->l1.d_inst);
  cudaFree(lay->l1.big);
  cudaFree(lay->l1.d_ids);
  cudaFree(lay->l1.mr_tw);
  cudaFree(lay->l1.mr_big);
  delete[] lay->l1.h_inst;
  sgn::batch2d_destroy(lay->b2);
  sgn::layout2d_destroy(lay->l2);
  cudaFree(lay->ws);
  cudaFree(lay->scratch);
  cudaFree(lay->coef_df);
  cudaFree(lay->rec);
  cudaFree(lay->given);
  delete lay;
}

extern "C" long long sgn_layout_points(const sgn_layout* lay) { return lay ? lay->points : -1; }

extern "C" sgn_status sgn_layout_set_forms(sgn_layout* lay, int log2n, int solve_ctas,
                                           int rhs_ctas) {
  auto bad = [](int c) { return c != 1 && c != 2; };
  if (check_layout(lay) || lay->dim != 1 || log2n < 3 || log2n > sgn::kMaxLog1d ||
      bad(solve_ctas) || bad(rhs_ctas))
    return fail(lay ? lay->ctx : nullptr, SGN_ERR_INVALID_ARG, "set_form args");
  for (int c : {solve_ctas, rhs_ctas})
    if ((c == 2 && log2n < sgn::kClusterLog1d) || (c == 1 && log2n > sgn::kSmemLog1d))
      return fail(lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "no such form for this size");
  sgn::Layout1d& L = lay->l1;
  if (L.ctas(log2n) != solve_ctas || L.rhs_ctas(log2n) != rhs_ctas) {
    L.form[log2n] = solve_ctas;
    L.rform[log2n] = rhs_ctas;
    L.gen += 1;
  }
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_set_form(sgn_layout* lay, int log2n, int ctas) {
  return sgn_layout_set_forms(lay, log2n, ctas, ctas);
}

extern "C" sgn_status sgn_layout_get_forms(const sgn_layout* lay, int log2n, int* solve_ctas,
                                           int* rhs_ctas) {
  if (check_layout(lay) || lay->dim != 1 || !solve_ctas || !rhs_ctas || log2n < 3 ||
      log2n > sgn::kMaxLog1d)
    return SGN_ERR_INVALID_ARG;
  *solve_ctas = lay->l1.ctas(log2n);
  *rhs_ctas = lay->l1.rhs_ctas(log2n);
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_get_form(const sgn_layout* lay, int log2n, int* ctas) {
  int r = 0;
  return sgn_layout_get_forms(lay, log2n, ctas, &r);
}

extern "C" sgn_status sgn_layout_set_form2d(sgn_layout* lay, int inner, int tile_width) {
  if (check_layout(lay) || lay->dim != 2 || (inner != 0 && inner != 1) ||
      (tile_width != 0 && tile_width != 1 && tile_width != 2 && tile_width != 4))
    return fail(lay ? lay->ctx : nullptr, SGN_ERR_INVALID_ARG, "set_form2d args");
  sgn::Layout2d& L = lay->l2;
  if (L.mr) return fail(lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "no inner-solve forms on this grid");
  const int tw = tile_width ? tile_width : sgn::persist2d_tile_width(L.nx, L.ny, 1, L.p_grid);
  if (!sgn::persist2d_tile_ok(L.nx, L.ny, tw))
    return fail(lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "tile width too wide for this grid");
  SGN_CUDA(lay->ctx, sgn::layout2d_set_inner_form(L, inner, tw));
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_set_radix2d(sgn_layout* lay, int max_radix) {
  if (check_layout(lay) || lay->dim != 2 || (max_radix != 0 && max_radix != 8 && max_radix != 16))
    return fail(lay ? lay->ctx : nullptr, SGN_ERR_INVALID_ARG, "set_radix2d args");
  if (lay->l2.mr) return fail(lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "no radix plans on this grid");
  SGN_CUDA(lay->ctx, sgn::layout2d_set_radix(lay->l2, max_radix == 16 ? 4 : 3));
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_set_unit_threads2d(sgn_layout* lay, int threads) {
  if (check_layout(lay) || lay->dim != 2 || (threads != 0 && threads != 128 && threads != 256))
    return fail(lay ? lay->ctx : nullptr, SGN_ERR_INVALID_ARG, "set_unit_threads2d args");
  if (lay->l2.mr) return fail(lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "no persistent solve on this grid");
  SGN_CUDA(lay->ctx, sgn::layout2d_set_unit_threads(lay->l2, threads));
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_get_unit_threads2d(const sgn_layout* lay, int* threads) {
  if (check_layout(lay) || lay->dim != 2 || !threads) return SGN_ERR_INVALID_ARG;
  *threads = lay->l2.p_gt;
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_get_radix2d(const sgn_layout* lay, int* max_radix) {
  if (check_layout(lay) || lay->dim != 2 || !max_radix) return SGN_ERR_INVALID_ARG;
  *max_radix = 1 << lay->l2.p_maxb;
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_get_form2d(const sgn_layout* lay, int* inner, int* tile_width) {
  if (check_layout(lay) || lay->dim != 2 || !inner || !tile_width) return SGN_ERR_INVALID_ARG;
  *inner = lay->l2.inner_form;
  *tile_width = lay->l2.p_tw;
  return SGN_OK;
}

extern "C" sgn_status sgn_layout_offsets(const sgn_layout* lay, long long* offsets) {
  if (!lay || !offsets) return SGN_ERR_INVALID_ARG;
  std::copy(lay->offsets.begin(), lay->offsets.end(), offsets);
  return SGN_OK;
}

// =======================================================================================
// Hot-path operations
// =======================================================================================

namespace {

sgn_status upload_given(sgn_layout* lay, const sgn_precond* P, cudaStream_t s) {
  std::vector<SolveRec> h(lay->count);
  for (int i = 0; i < lay->count; ++i) {
    SolveRec r = {};
    r.sigma = P[i].sigma;
    r.alpha = P[i].alpha;
    r.kappa_ub = P[i].kappa_ub;
    r.flat = P[i].flat;
    if (!(r.sigma > 0.0) || !(r.alpha > 0.0))
      return fail(lay->ctx, SGN_ERR_INVALID_ARG, "preconditioner sigma, alpha must be > 0");
    h[i] = r;
  }
  SGN_CUDA(lay->ctx, cudaMemcpyAsync(lay->given, h.data(), sizeof(SolveRec) * lay->count,
                                     cudaMemcpyHostToDevice, s));
  // pageable source: the copy is staged before return, but keep `h` alive until it lands
  SGN_CUDA(lay->ctx, cudaStreamSynchronize(s));
  return SGN_OK;
}

sgn_status fetch_recs(sgn_layout* lay, std::vector<SolveRec>& h, cudaStream_t s) {
  h.resize(lay->count);
  SGN_CUDA(lay->ctx, cudaMemcpyAsync(h.data(), lay->rec, sizeof(SolveRec) * lay->count,
                                     cudaMemcpyDeviceToHost, s));
  SGN_CUDA(lay->ctx, cudaStreamSynchronize(s));
  return SGN_OK;
}

}  // namespace

namespace {

bool is_batch2d(const sgn_layout* lay) { return lay->dim == 2 && lay->count > 1; }

// A single-instance 2d operation over every instance of a 2d batch: instance b's fields are
// staged into its block st (eta [P], vector 0 [2P], vector 1 [2P], output [2P], in the
// single-instance packing), op(L_b, st, b) runs, and the output vector goes back to `out`.
template <typename Op>
cudaError_t each_instance2d(sgn_layout* lay, const double* scal, const double* v0,
                            const double* v1, double* out, cudaStream_t s, Op op) {
  sgn::Batch2d& Bt = lay->b2;
  const long long P = lay->l2.P, Ptot = lay->points;
  cudaError_t e;
  for (int b = 0; b < Bt.B; ++b) {
    double* st = Bt.stage + 7 * P * b;
    sgn::Layout2d& L = Bt.inst(lay->l2, b);
    if ((e = sgn::batch2d_stage_in(L, st, b, Ptot, scal, v0, v1, nullptr, s)) ||
        (e = op(L, st, b)))
      return e;
    if (out && (e = sgn::batch2d_stage_out(L, st + 5 * P, b, Ptot, out, s))) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" sgn_status sgn_spectral_grad(sgn_ctx* ctx, const sgn_layout* lay_c, const double* f,
                                        double* gradf, sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !f || !gradf) return fail(ctx, SGN_ERR_INVALID_ARG, "grad");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e =
      lay->dim == 1 ? sgn::launch_deriv1d(lay->l1, ctx->tw64, f, gradf, s)
      : is_batch2d(lay)
          ? each_instance2d(lay, f, nullptr, nullptr, gradf, s,
                            [&](sgn::Layout2d& L, double* st, int) {
                              return sgn::launch_grad2d(L, ctx->tw64, st, st + 5 * L.P, s);
                            })
          : sgn::launch_grad2d(lay->l2, ctx->tw64, f, gradf, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sgn_spectral_grad");
  return SGN_OK;
}

extern "C" sgn_status sgn_precond_coeffs(sgn_ctx* ctx, const sgn_layout* lay_c, const double* eta,
                                         const double* gradh, sgn_coef_kind kind,
                                         sgn_precond* out, sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !eta || !gradh || !out)
    return fail(ctx, SGN_ERR_INVALID_ARG, "coeffs");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e =
      lay->dim == 1 ? sgn::launch_coeffs1d(lay->l1, eta, gradh, kind, lay->rec, s)
      : is_batch2d(lay)
          ? each_instance2d(lay, eta, gradh, nullptr, nullptr, s,
                            [&](sgn::Layout2d& L, double* st, int b) {
                              return sgn::launch_coeffs2d(L, st, st + L.P, kind, lay->rec + b, s);
                            })
          : sgn::launch_coeffs2d(lay->l2, eta, gradh, kind, lay->rec, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sgn_precond_coeffs");
  std::vector<SolveRec> h;
  sgn_status st = fetch_recs(lay, h, s);
  if (st) return st;
  sgn_status worst = SGN_OK;
  for (int i = 0; i < lay->count; ++i) {
    out[i].sigma = h[i].sigma;
    out[i].alpha = h[i].alpha;
    out[i].kappa_ub = h[i].kappa_ub;
    out[i].flat = h[i].flat;
    if (h[i].status != SGN_OK) worst = (sgn_status)h[i].status;
  }
  if (worst != SGN_OK) return fail(ctx, worst, "non-positive depth in some instance");
  return SGN_OK;
}

extern "C" sgn_status sgn_apply_operator(sgn_ctx* ctx, const sgn_layout* lay_c, const double* eta,
                                         const double* gradh, const double* u, double* Gu,
                                         sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !eta || !gradh || !u || !Gu)
    return fail(ctx, SGN_ERR_INVALID_ARG, "apply_operator");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  cudaError_t e =
      lay->dim == 1 ? sgn::launch_apply_G1d(lay->l1, ctx->tw64, eta, gradh, u, Gu, s)
      : is_batch2d(lay)
          ? each_instance2d(lay, eta, gradh, u, Gu, s,
                            [&](sgn::Layout2d& L, double* st, int) {
                              const long long P = L.P;
                              return sgn::launch_apply_G2d(L, ctx->tw64, st, st + P, st + 3 * P,
                                                           st + 5 * P, s);
                            })
          : sgn::launch_apply_G2d(lay->l2, ctx->tw64, eta, gradh, u, Gu, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sgn_apply_operator");
  return SGN_OK;
}

extern "C" sgn_status sgn_precond_solve(sgn_ctx* ctx, const sgn_layout* lay_c,
                                        const sgn_precond* P, const double* r, double* z,
                                        sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !P || !r || !z)
    return fail(ctx, SGN_ERR_INVALID_ARG, "precond_solve");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  sgn_status st = upload_given(lay, P, s);
  if (st) return st;
  cudaError_t e =
      lay->dim == 1 ? sgn::launch_precond1d(lay->l1, ctx->tw64, lay->given, r, z, s)
      : is_batch2d(lay)
          ? each_instance2d(lay, nullptr, nullptr, r, z, s,
                            [&](sgn::Layout2d& L, double* st, int b) {
                              return sgn::launch_precond2d(L, ctx->tw64, lay->given + b,
                                                           st + 3 * L.P, st + 5 * L.P, s);
                            })
          : sgn::launch_precond2d(lay->l2, ctx->tw64, lay->given, r, z, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sgn_precond_solve");
  return SGN_OK;
}

namespace {

sgn_status run_pcg(sgn_layout* lay, const double* eta, const double* gradh, const SolveRec* given,
                   sgn_coef_kind kind, const double* b, double* x, double rtol, int maxit,
                   sgn_precision prec, double rtol_inner, int max_refine, cudaStream_t s) {
  sgn_ctx* ctx = lay->ctx;
  if (rtol_inner <= 0.0) rtol_inner = -1.0;   // adaptive inner tolerance
  if (max_refine <= 0) max_refine = 12;
  cudaError_t e;
  ProfScope prof(ctx, s, 0);
  if (lay->dim == 1) {
    e = sgn::launch_pcg1d(lay->l1, ctx->tw64, ctx->tw32, prec, eta, gradh, b, x, given, kind, rtol,
                          rtol_inner, maxit, max_refine, lay->rec, lay->ws, lay->coef_df, s);
  } else if (lay->count > 1) {
    e = sgn::launch_pcg2d_batch(lay->l2, lay->b2, ctx->tw64, ctx->tw32, prec, eta, gradh, b, x,
                                given, kind, rtol, rtol_inner, maxit, max_refine, lay->rec, s);
  } else {
    e = sgn::launch_pcg2d(lay->l2, ctx->tw64, ctx->tw32, prec, eta, gradh, b, x, given, kind, rtol,
                          rtol_inner, maxit, max_refine, lay->rec, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pcg launch");
  return SGN_OK;
}

}  // namespace

extern "C" sgn_status sgn_pcg(sgn_ctx* ctx, const sgn_layout* lay_c, const double* eta,
                              const double* gradh, const sgn_precond* P, const double* b,
                              double* x, double rtol, int maxit, sgn_precision prec,
                              sgn_pcg_info* info, sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !eta || !gradh || !b || !x || !(rtol > 0.0) || maxit < 0 ||
      (prec != SGN_PREC_FP64 && prec != SGN_PREC_MIXED))
    return fail(ctx, SGN_ERR_INVALID_ARG, "pcg args");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  const SolveRec* given = nullptr;
  if (P) {
    sgn_status st = upload_given(lay, P, s);
    if (st) return st;
    given = lay->given;
  }
  sgn_status st = run_pcg(lay, eta, gradh, given, SGN_COEF_OPT, b, x, rtol, maxit, prec, 0.0, 0, s);
  if (st) return st;
  if (!info) return SGN_OK;
  std::vector<SolveRec> h;
  st = fetch_recs(lay, h, s);
  if (st) return st;
  sgn_status worst = SGN_OK;
  for (int i = 0; i < lay->count; ++i) {
    info[i].iters = h[i].iters;
    info[i].refinements = h[i].refinements;
    info[i].rel_resid_Ainv = h[i].ratio;
    info[i].status = h[i].status;
    if (h[i].status > worst) worst = (sgn_status)h[i].status;
  }
  if (worst != SGN_OK) return fail(ctx, worst, "pcg: some instance did not finish cleanly");
  return SGN_OK;
}

namespace {

// The solve report of every instance in the ABI's sgn_pcg_info form, on the device.
__global__ void k_pcg_info(const SolveRec* __restrict__ rec, sgn_pcg_info* __restrict__ info,
                           int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const SolveRec r = rec[i];
  sgn_pcg_info o;
  o.iters = r.iters;
  o.refinements = r.refinements;
  o.rel_resid_Ainv = r.ratio;
  o.status = r.status;
  info[i] = o;
}

}  // namespace

extern "C" sgn_status sgn_pcg_async(sgn_ctx* ctx, const sgn_layout* lay_c, const double* eta,
                                    const double* gradh, const double* b, double* x, double rtol,
                                    int maxit, sgn_precision prec, sgn_pcg_info* info,
                                    sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !eta || !gradh || !b || !x || !info || !(rtol > 0.0) ||
      maxit < 0 || (prec != SGN_PREC_FP64 && prec != SGN_PREC_MIXED))
    return fail(ctx, SGN_ERR_INVALID_ARG, "pcg_async args");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  sgn_status st = run_pcg(lay, eta, gradh, nullptr, SGN_COEF_OPT, b, x, rtol, maxit, prec, 0.0, 0, s);
  if (st) return st;
  k_pcg_info<<<(lay->count + 127) / 128, 128, 0, s>>>(lay->rec, info, lay->count);
  SGN_CUDA(ctx, cudaGetLastError());
  return SGN_OK;
}

extern "C" sgn_status sgn_gmres(sgn_ctx* ctx, const sgn_layout* lay_c, const double* eta,
                                const double* gradh, const sgn_precond* P, const double* b,
                                double* x, double rtol, int restart, int maxit,
                                sgn_pcg_info* info, sgn_stream stream) {
  sgn_layout* lay = const_cast<sgn_layout*>(lay_c);
  if (!ctx || check_layout(lay) || !eta || !gradh || !b || !x || !(rtol > 0.0) || maxit < 0 ||
      restart < 1 || restart > SGN_GMRES_MAX_RESTART)
    return fail(ctx, SGN_ERR_INVALID_ARG, "gmres args");
  if (is_batch2d(lay)) return fail(ctx, SGN_ERR_INVALID_ARG, "gmres on a 2d batch");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  sgn::GmresArgs a;
  if (P) {
    sgn_status st = upload_given(lay, P, s);
    if (st) return st;
    a.coef = lay->given;
  } else {
    cudaError_t e = lay->dim == 1
                        ? sgn::launch_coeffs1d(lay->l1, eta, gradh, SGN_COEF_OPT, lay->rec, s)
                        : sgn::launch_coeffs2d(lay->l2, eta, gradh, SGN_COEF_OPT, lay->rec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gmres coefficients");
    a.coef = lay->rec;
  }
  a.dim = lay->dim;
  a.count = lay->count;
  a.l1 = &lay->l1;
  a.l2 = &lay->l2;
  a.offsets = lay->offsets.data();
  a.vec_len = (long long)lay->dim * lay->points;
  a.tw64 = ctx->tw64;
  a.eta = eta;
  a.gradh = gradh;
  a.b = b;
  a.x = x;
  a.rec = lay->rec;
  a.rtol = rtol;
  a.restart = restart;
  a.maxit = maxit;
  cudaError_t e = sgn::run_gmres(a, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gmres");
  std::vector<SolveRec> h;
  sgn_status st = fetch_recs(lay, h, s);
  if (st) return st;
  sgn_status worst = SGN_OK;
  for (int i = 0; i < lay->count; ++i) {
    if (info) {
      info[i].iters = h[i].iters;
      info[i].refinements = h[i].refinements;
      info[i].rel_resid_Ainv = h[i].ratio;
      info[i].status = h[i].status;
    }
    if (h[i].status > worst) worst = (sgn_status)h[i].status;
  }
  if (worst != SGN_OK) return fail(ctx, worst, "gmres: some instance did not finish cleanly");
  return SGN_OK;
}

extern "C" sgn_status sgn_rhs(sgn_ctx* ctx, const sgn_layout* lay, const double* eta,
                              const double* u, const double* h, const double* gradh,
                              double* f_eta, double* f_U, sgn_stream stream) {
  if (!ctx || check_layout(lay) || !eta || !u || !h || !gradh || !f_eta || !f_U)
    return fail(ctx, SGN_ERR_INVALID_ARG, "rhs args");
  if (is_batch2d(lay)) return fail(ctx, SGN_ERR_INVALID_ARG, "rhs on a 2d batch");
  DeviceGuard g(ctx->device);
  const double grav = lay->grids[0].g;
  ProfScope prof(ctx, as_stream(stream), 1);
  cudaError_t e =
      lay->dim == 1
          ? sgn::launch_rhs1d(lay->l1, ctx->tw64, ctx->tw32, SGN_PREC_FP64, grav, eta, u, h, gradh,
                              f_eta, f_U, lay->scratch, as_stream(stream))
          : sgn::launch_rhs2d(lay->l2, ctx->tw64, ctx->tw32, SGN_PREC_FP64, grav, eta, u, h,
                              gradh, f_eta, f_U, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sgn_rhs");
  return SGN_OK;
}

// =======================================================================================
// Time integration
// =======================================================================================

enum HistKind { HIST_NONE = 0, HIST_AB = 1, HIST_SBDF2 = 2 };

struct sgn_state {
  sgn_layout* lay = nullptr;
  double* eta = nullptr;
  double* U = nullptr;
  double* u = nullptr;
  const double* h = nullptr;
  double* gradh = nullptr;
  int d = 1;                        // components of a vector field
  long long P = 0;
  // library-owned workspace (each array d*P or P doubles)
  std::vector<double*> bufs;
  double* fe[4] = {nullptr};        // RK4 stage right-hand sides
  double* fU[4] = {nullptr};
  double* he[4] = {nullptr};        // multistep history (oldest first)
  double* hU[4] = {nullptr};
  double* eta_s = nullptr;
  double* U_s = nullptr;
  double* u_s = nullptr;
  double* eta_p = nullptr;          // SBDF2 previous level
  double* U_p = nullptr;
  double* ut = nullptr;             // non-constraint form: the last u_t (next warm start)
  // RK4 history for the first stage solve's starting point: u at the start of the last RK4
  // step (u_prev) and the u that step returned (u_last; NaN when there is none)
  double* u_prev = nullptr;
  double* u_last = nullptr;
  void* res0 = nullptr;             // SBDF2 residual spectra (previous / current)
  void* res1 = nullptr;
  double* dt_dev = nullptr;
  double* t_dev = nullptr;          // per-instance simulated time (external forcing)
  ForceTerms force{};               // external forcing (K = 0: none)
  SolveRec* A_fixed = nullptr;      // SBDF2 preconditioner, fixed at init
  DevStats* stats = nullptr;
  int hist = HIST_NONE;
  int dealias = 0;                  // 2/3-rule projection of every new level
  int levels = 0;                   // valid multistep levels
  int prec = SGN_PREC_FP64;         // precision of the current step call
  std::vector<double> dt_last;
  double t = 0.0;
  long long step = 0;
  cudaStream_t last = nullptr;
  // CUDA graph of one 1d RK4 step, replayed while the step options repeat
  cudaStream_t gs = nullptr;        // capture / replay stream (joined to the caller's by events)
  cudaEvent_t ge0 = nullptr, ge1 = nullptr;
  cudaGraph_t graph = nullptr;      // the captured graph (its nodes address gexec's nodes)
  cudaGraphExec_t gexec = nullptr;
  std::vector<CapRec> gprof;        // profiled launch groups of gexec
  sgn_opts gkey{};                  // options of the last 1d RK4 step
  int gkey_prof = -1;               // profiling state it was taken with (-1: none yet)
  int gkey_gen = -1;                // the layout's kernel forms it was taken with
  bool gdisabled = false;           // capture failed once: direct launches from then on
};

namespace {

sgn_status alloc_state(sgn_state* st) {
  const long long P = st->P;
  const long long V = st->d * P;
  auto get = [&](long long n) -> double* {
    double* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * (size_t)std::max<long long>(n, 1)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    st->bufs.push_back(p);
    return p;
  };
  for (int i = 0; i < 4; ++i) {
    if (!(st->fe[i] = get(P)) || !(st->fU[i] = get(V)) || !(st->he[i] = get(P)) ||
        !(st->hU[i] = get(V)))
      return SGN_ERR_NOMEM;
  }
  if (!(st->eta_s = get(P)) || !(st->U_s = get(V)) || !(st->u_s = get(V)) ||
      !(st->eta_p = get(P)) || !(st->U_p = get(V)) || !(st->ut = get(V)) ||
      !(st->u_prev = get(V)) || !(st->u_last = get(V)) ||
      !(st->dt_dev = get(st->lay->count)) || !(st->t_dev = get(st->lay->count)))
    return SGN_ERR_NOMEM;
  const size_t res_bytes = st->lay->dim == 1 ? sizeof(double) * 2 * (size_t)(st->lay->l1.ws_cplx /
                                                                            sgn::kWsVectors)
                                             : sgn::layout2d_res_bytes(st->lay->l2);
  // no RK4 history yet: NaN compares unequal to every u
  if (cudaMemset(st->u_last, 0xff, sizeof(double) * (size_t)std::max<long long>(V, 1)) !=
      cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_NOMEM;
  }
  if (cudaMalloc(&st->res0, res_bytes) != cudaSuccess ||
      cudaMalloc(&st->res1, res_bytes) != cudaSuccess ||
      cudaMalloc(&st->A_fixed, sizeof(SolveRec) * st->lay->count) != cudaSuccess ||
      cudaMalloc(&st->stats, sizeof(DevStats)) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_NOMEM;
  }
  return SGN_OK;
}

sgn_status upload_dt(sgn_state* st, const double* dt, cudaStream_t s) {
  for (int i = 0; i < st->lay->count; ++i)
    if (!(dt[i] > 0.0)) return fail(st->lay->ctx, SGN_ERR_INVALID_ARG, "dt must be > 0");
  bool same = (int)st->dt_last.size() == st->lay->count &&
              std::equal(st->dt_last.begin(), st->dt_last.end(), dt);
  if (!same) {
    st->dt_last.assign(dt, dt + st->lay->count);
    SGN_CUDA(st->lay->ctx, cudaMemcpyAsync(st->dt_dev, st->dt_last.data(),
                                           sizeof(double) * st->lay->count,
                                           cudaMemcpyHostToDevice, s));
    SGN_CUDA(st->lay->ctx, cudaStreamSynchronize(s));
  }
  return SGN_OK;
}

using Terms = std::initializer_list<std::pair<const double*, double>>;

LinComb make_lincomb(Terms xs, Terms fs) {
  LinComb lc{};
  for (auto& p : xs) {
    lc.x[lc.nx] = p.first;
    lc.a[lc.nx] = p.second;
    ++lc.nx;
  }
  for (auto& p : fs) {
    lc.f[lc.nf] = p.first;
    lc.c[lc.nf] = p.second;
    ++lc.nf;
  }
  return lc;
}

// Starting point of a time step's first solve (reading R8): at every point where u is still
// the value the last step of this state returned, u + c (u - u_prev), the linear
// extrapolation from that step's start (c = 1/2: the RK4 stage at t + dt/2; c = 1: the AB
// solve at t + dt), an O(dt^2) guess in place of u's O(dt); elsewhere (no history, or u
// changed since) u itself.  Only the solve's starting point depends on it; its stopping
// rule is unchanged.
__global__ void k_step_guess(long long n, double c, const double* __restrict__ u,
                             const double* __restrict__ u_last,
                             const double* __restrict__ u_prev, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = u[i];
    out[i] = v == u_last[i] ? v + c * (v - u_prev[i]) : v;
  }
}

// out = sum a_t x_t + dt sum c_t f_t for scalar (components=1) or vector fields; with out2
// set, a second combination in the same launch (1d) or right after it (2d)
sgn_status lincomb(sgn_state* st, double* out, Terms xs, Terms fs, int components,
                   cudaStream_t s, double* out2 = nullptr, Terms xs2 = {}, Terms fs2 = {},
                   int components2 = 0) {
  const LinComb lc = make_lincomb(xs, fs), lc2 = make_lincomb(xs2, fs2);
  if (st->lay->dim == 1) {
    const sgn::Layout1d& L = st->lay->l1;
    const int maxn = L.maxn;
    LinJobs J{};
    J.j[0] = LinJob{out, lc, components};
    J.j[1] = LinJob{out2, lc2, components2};
    const dim3 grid((maxn + kLinChunk - 1) / kLinChunk, L.count, out2 ? 2 : 1);
    k_lincomb<<<grid, 256, 0, s>>>(L.d_inst, st->dt_dev, J, st->P);
  } else {
    sgn::launch_lincomb2d(st->lay->l2, st->dt_dev, out, lc.x, lc.a, lc.nx, lc.f, lc.c, lc.nf,
                          components, s);
    if (out2)
      sgn::launch_lincomb2d(st->lay->l2, st->dt_dev, out2, lc2.x, lc2.a, lc2.nx, lc2.f, lc2.c,
                            lc2.nf, components2, s);
  }
  SGN_CUDA(st->lay->ctx, cudaGetLastError());
  return SGN_OK;
}

// fe, fU += the external forcing at the stage time t_i + c dt_i (nothing when unset)
sgn_status force_at(sgn_state* st, double* fe, double* fU, double c, cudaStream_t s) {
  if (st->force.K == 0) return SGN_OK;
  const bool d1 = st->lay->dim == 1;
  int maxn = 8;
  long long n2d = 0;
  if (d1) {
    maxn = st->lay->l1.maxn;
  } else {
    n2d = st->P;
  }
  const long long span = d1 ? maxn : n2d;
  const dim3 grid((unsigned)((span + kLinChunk - 1) / kLinChunk), st->lay->count, 1);
  k_force<<<grid, 256, 0, s>>>(d1 ? st->lay->l1.d_inst : nullptr, st->t_dev, st->dt_dev, c,
                               st->force, fe, fU, st->P, st->d, n2d);
  SGN_CUDA(st->lay->ctx, cudaGetLastError());
  return SGN_OK;
}

sgn_status advance_time(sgn_state* st, cudaStream_t s) {
  if (st->force.K == 0) return SGN_OK;
  k_advance_time<<<1, 256, 0, s>>>(st->t_dev, st->dt_dev, st->lay->count);
  SGN_CUDA(st->lay->ctx, cudaGetLastError());
  return SGN_OK;
}

sgn_status rhs_plain(sgn_state* st, const double* eta, const double* u, double* fe, double* fU,
                     cudaStream_t s);

// Right-hand side inside the steppers (float64 for FP64 solves, double-float for MIXED),
// plus the external forcing at the stage time t + c dt.
sgn_status rhs_at(sgn_state* st, const double* eta, const double* u, double* fe, double* fU,
                  cudaStream_t s, double c = 0.0) {
  const sgn_status r = rhs_plain(st, eta, u, fe, fU, s);
  if (r != SGN_OK) return r;
  return force_at(st, fe, fU, c, s);
}

// With dealiasing on, a new time level is projected by the 2/3 rule before anything is
// computed from it: eta - h and U, and u where it is not solved from U (SBDF2); 1d transforms
// in the precision of the step (double-float on the mixed path), 2d in float64.
sgn_status dealias_at(sgn_state* st, double* eta, double* U, double* u, cudaStream_t s) {
  if (!st->dealias) return SGN_OK;
  sgn_ctx* ctx = st->lay->ctx;
  const cudaError_t e =
      st->lay->dim == 1 ? sgn::launch_dealias1d(st->lay->l1, ctx->tw64, ctx->tw32, st->prec,
                                                st->h, eta, U, u, s)
                        : sgn::launch_dealias2d(st->lay->l2, ctx->tw64, st->h, eta, U, u, s);
  if (e != cudaSuccess) return cuda_fail(st->lay->ctx, e, "dealias launch");
  return SGN_OK;
}

sgn_status rhs_plain(sgn_state* st, const double* eta, const double* u, double* fe, double* fU,
                     cudaStream_t s) {
  sgn_layout* lay = st->lay;
  if (st->prec != SGN_PREC_MIXED) return sgn_rhs(lay->ctx, lay, eta, u, st->h, st->gradh, fe, fU, s);
  if (lay->dim == 2) {
    ProfScope prof(lay->ctx, s, 1);
    const cudaError_t e = sgn::launch_rhs2d(lay->l2, lay->ctx->tw64, lay->ctx->tw32,
                                            SGN_PREC_MIXED, lay->grids[0].g, eta, u, st->h,
                                            st->gradh, fe, fU, s);
    if (e != cudaSuccess) return cuda_fail(lay->ctx, e, "rhs launch");
    return SGN_OK;
  }
  ProfScope prof(lay->ctx, s, 1);
  cudaError_t e = sgn::launch_rhs1d(lay->l1, lay->ctx->tw64, lay->ctx->tw32, SGN_PREC_MIXED,
                                    lay->grids[0].g, eta, u, st->h, st->gradh, fe, fU,
                                    lay->scratch, s);
  if (e != cudaSuccess) return cuda_fail(lay->ctx, e, "rhs launch");
  return SGN_OK;
}

sgn_status solve_at(sgn_state* st, const double* eta, const double* U, double* u,
                    const sgn_opts* o, cudaStream_t s) {
  sgn_status r = run_pcg(st->lay, eta, st->gradh, nullptr, o->coef, U, u, o->rtol, o->maxit,
                         o->prec, o->rtol_inner, o->max_refine, s);
  if (r) return r;
  const bool d1 = st->lay->dim == 1;
  k_accum<<<1, 256, 0, s>>>(st->lay->rec, d1 ? st->lay->l1.d_inst : nullptr, st->lay->count,
                           d1 ? 0 : st->lay->l2.P, d1 ? 0 : st->lay->l2.lx + st->lay->l2.ly,
                           o->prec == SGN_PREC_MIXED, st->stats);
  SGN_CUDA(st->lay->ctx, cudaGetLastError());
  return SGN_OK;
}

sgn_status copy_field(sgn_state* st, double* dst, const double* src, long long n, cudaStream_t s) {
  SGN_CUDA(st->lay->ctx, cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return SGN_OK;
}

#define SGN_TRY(expr)            \
  do {                           \
    sgn_status s_ = (expr);      \
    if (s_ != SGN_OK) return s_; \
  } while (0)

// Solve G u = U at eta, then the right-hand side at (eta, u).  For 1d layouts the
// right-hand side reuses the u_x that the solve leaves in the scratch planes.
sgn_status stage_at(sgn_state* st, const double* eta, const double* U, double* u, double* fe,
                    double* fU, const sgn_opts* o, cudaStream_t s, double c) {
  sgn_layout* lay = st->lay;
  if (lay->dim != 1) {
    SGN_TRY(solve_at(st, eta, U, u, o, s));
    return rhs_at(st, eta, u, fe, fU, s, c);
  }
  sgn_ctx* ctx = lay->ctx;
  const double rtol_inner = o->rtol_inner > 0.0 ? o->rtol_inner : -1.0;
  const int max_refine = o->max_refine > 0 ? o->max_refine : 12;
  {
    ProfScope prof(ctx, s, 0);
    const cudaError_t e = sgn::launch_pcg1d_ux(
        lay->l1, ctx->tw64, ctx->tw32, o->prec, eta, st->gradh, U, u, o->coef, o->rtol,
        rtol_inner, o->maxit, max_refine, lay->rec, lay->ws, lay->coef_df, lay->scratch, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pcg launch");
  }
  k_accum<<<1, 256, 0, s>>>(lay->rec, lay->l1.d_inst, lay->count, 0, 0,
                           o->prec == SGN_PREC_MIXED, st->stats);
  SGN_CUDA(ctx, cudaGetLastError());
  ProfScope prof(ctx, s, 1);
  const cudaError_t e = sgn::launch_rhs1d_ux(lay->l1, ctx->tw64, ctx->tw32, o->prec,
                                             lay->grids[0].g, eta, u, st->h, st->gradh, fe, fU,
                                             lay->scratch, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rhs launch");
  return force_at(st, fe, fU, c, s);
}

// One RK4 step (Eq:ERK): stages with a_{i,i-1} = 1/2, 1/2, 1 and weights 1/6, 1/3, 1/3, 1/6.
// u_s = the first solve's starting point (k_step_guess, c as there)
sgn_status step_guess(sgn_state* st, double c, double* out, cudaStream_t s) {
  const long long V = (long long)st->d * st->P;
  const long long nb = std::min<long long>((V + 255) / 256, 4096);
  k_step_guess<<<(int)std::max<long long>(nb, 1), 256, 0, s>>>(V, c, st->u, st->u_last,
                                                                st->u_prev, out);
  SGN_CUDA(st->lay->ctx, cudaGetLastError());
  return SGN_OK;
}

sgn_status rk4_once(sgn_state* st, const sgn_opts* o, cudaStream_t s) {
  const int d = st->d;
  const long long P = st->P, V = d * P;
  static const double a[4] = {0.0, 0.5, 0.5, 1.0};
  SGN_TRY(rhs_at(st, st->eta, st->u, st->fe[0], st->fU[0], s));
  SGN_TRY(step_guess(st, 0.5, st->u_s, s));
  for (int i = 1; i < 4; ++i) {
    SGN_TRY(lincomb(st, st->eta_s, {{st->eta, 1.0}}, {{st->fe[i - 1], a[i]}}, 1, s, st->U_s,
                    {{st->U, 1.0}}, {{st->fU[i - 1], a[i]}}, d));
    // stage 4 (c = 1) starts from u extrapolated from c = 0 and c = 1/2: 2 u^(3) - u_n
    // (only the initial guess of the solve changes)
    if (i == 3) SGN_TRY(lincomb(st, st->u_s, {{st->u_s, 2.0}, {st->u, -1.0}}, {}, d, s));
    SGN_TRY(stage_at(st, st->eta_s, st->U_s, st->u_s, st->fe[i], st->fU[i], o, s, a[i]));
  }
  const double b0 = 1.0 / 6.0, b1 = 1.0 / 3.0;
  SGN_TRY(lincomb(st, st->eta, {{st->eta, 1.0}},
                  {{st->fe[0], b0}, {st->fe[1], b1}, {st->fe[2], b1}, {st->fe[3], b0}}, 1, s,
                  st->U, {{st->U, 1.0}},
                  {{st->fU[0], b0}, {st->fU[1], b1}, {st->fU[2], b1}, {st->fU[3], b0}}, d));
  SGN_TRY(dealias_at(st, st->eta, st->U, nullptr, s));
  SGN_TRY(copy_field(st, st->u_prev, st->u, V, s));        // u at this step's start
  SGN_TRY(copy_field(st, st->u, st->u_s, V, s));
  SGN_TRY(solve_at(st, st->eta, st->U, st->u, o, s));
  SGN_TRY(copy_field(st, st->u_last, st->u, V, s));        // the u this step returns
  SGN_TRY(advance_time(st, s));
  (void)P;
  st->t += st->dt_last[0];
  st->step += 1;
  return SGN_OK;
}

sgn_status check_opts(sgn_state* st, const sgn_opts* o) {
  if (!o || !(o->rtol > 0.0) || o->maxit <= 0 ||
      (o->prec != SGN_PREC_FP64 && o->prec != SGN_PREC_MIXED))
    return fail(st->lay->ctx, SGN_ERR_INVALID_ARG, "opts");
  st->prec = o->prec;
  return SGN_OK;
}

}  // namespace

extern "C" sgn_status sgn_state_create(sgn_ctx* ctx, const sgn_layout* lay, double* eta, double* U,
                                       double* u, const double* h, double* gradh,
                                       sgn_state** out) {
  if (!ctx || check_layout(lay) || !eta || !U || !u || !h || !gradh || !out)
    return fail(ctx, SGN_ERR_INVALID_ARG, "state args");
  if (is_batch2d(lay)) return fail(ctx, SGN_ERR_INVALID_ARG, "states on a 2d batch");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  sgn_state* st = new (std::nothrow) sgn_state();
  if (!st) return SGN_ERR_NOMEM;
  st->lay = const_cast<sgn_layout*>(lay);
  st->eta = eta;
  st->U = U;
  st->u = u;
  st->h = h;
  st->gradh = gradh;
  st->d = lay->dim;
  st->P = lay->points;
  sgn_status r = alloc_state(st);
  if (r) {
    sgn_state_free(st);
    return fail(ctx, r, "state allocation");
  }
  *out = st;
  return SGN_OK;
}

extern "C" sgn_status sgn_state_init(sgn_state* st, sgn_stream stream) {
  if (!st) return SGN_ERR_INVALID_ARG;
  sgn_ctx* ctx = st->lay->ctx;
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  SGN_TRY(sgn_spectral_grad(ctx, st->lay, st->h, st->gradh, stream));
  SGN_TRY(sgn_apply_operator(ctx, st->lay, st->eta, st->gradh, st->u, st->U, stream));
  cudaError_t e = st->lay->dim == 1
                      ? sgn::launch_coeffs1d(st->lay->l1, st->eta, st->gradh, SGN_COEF_OPT,
                                             st->A_fixed, s)
                      : sgn::launch_coeffs2d(st->lay->l2, st->eta, st->gradh, SGN_COEF_OPT,
                                             st->A_fixed, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state init coefficients");
  SGN_CUDA(ctx, cudaMemsetAsync(st->stats, 0, sizeof(DevStats), s));
  SGN_CUDA(ctx, cudaMemsetAsync(st->t_dev, 0, sizeof(double) * st->lay->count, s));
  SGN_CUDA(ctx, cudaMemsetAsync(st->ut, 0, sizeof(double) * st->d * st->P, s));
  // the RK4 history starts over (NaN compares unequal to every u)
  SGN_CUDA(ctx, cudaMemsetAsync(st->u_last, 0xff, sizeof(double) * st->d * st->P, s));
  st->hist = HIST_NONE;
  st->levels = 0;
  st->t = 0.0;
  st->step = 0;
  st->last = s;
  return SGN_OK;
}

// Internal (serving): treat the bound arrays as a state that is already initialised (its
// gradh and U were computed earlier, for example per request before packing into a
// batch); clear counters and multistep history only.
namespace sgn {
// The RK4 history arrays of a state (d P doubles each; see k_rk4_guess), for callers that
// pack a request's state into a shared batched state and back (the server).
double* state_rk4_prev(sgn_state* st) { return st->u_prev; }
double* state_rk4_last(sgn_state* st) { return st->u_last; }

sgn_status state_attach(sgn_state* st, cudaStream_t s) {
  if (!st) return SGN_ERR_INVALID_ARG;
  DeviceGuard g(st->lay->device);
  SGN_CUDA(st->lay->ctx, cudaMemsetAsync(st->stats, 0, sizeof(DevStats), s));
  st->hist = HIST_NONE;
  st->levels = 0;
  st->last = s;
  return SGN_OK;
}
}  // namespace sgn

namespace {

void graph_drop(sgn_state* st) {
  if (st->gexec) cudaGraphExecDestroy(st->gexec);
  if (st->graph) cudaGraphDestroy(st->graph);
  st->gexec = nullptr;
  st->graph = nullptr;
  st->gprof.clear();
}

bool same_opts(const sgn_opts& a, const sgn_opts& b) {
  return a.rtol == b.rtol && a.maxit == b.maxit && a.prec == b.prec && a.coef == b.coef &&
         a.rtol_inner == b.rtol_inner && a.max_refine == b.max_refine;
}

// Captures one RK4 step of a 1d state into st->gexec (launch work only: every array and the
// per-instance dt are device buffers of the state, so one graph serves every later step).
sgn_status graph_capture(sgn_state* st, const sgn_opts* o) {
  sgn_ctx* ctx = st->lay->ctx;
  if (!st->gs && (cudaStreamCreateWithFlags(&st->gs, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&st->ge0, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&st->ge1, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  std::vector<CapRec> prof;
  const double t0 = st->t;
  const long long k0 = st->step;
  if (cudaStreamBeginCapture(st->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  ctx->capture = ctx->prof ? &prof : nullptr;
  const sgn_status r = rk4_once(st, o, st->gs);
  ctx->capture = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st->gs, &graph);
  st->t = t0;                       // the capture ran nothing
  st->step = k0;
  cudaGraphExec_t exec = nullptr;
  const bool ok = r == SGN_OK && ec == cudaSuccess && graph &&
                  cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) ==
                      cudaSuccess &&
                  (!ctx->prof || prof.size() > 0);
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  st->graph = graph;
  st->gexec = exec;
  st->gprof = std::move(prof);
  return SGN_OK;
}

// One replay on st->gs, ordered after the caller's prior work on s and before its later work.
sgn_status graph_replay(sgn_state* st, cudaStream_t s) {
  sgn_ctx* ctx = st->lay->ctx;
  if (ctx->prof) {
    for (const CapRec& c : st->gprof) {
      ProfRec r{};
      r.kind = c.kind;
      auto take = [&]() {
        cudaEvent_t e;
        if (!ctx->pool.empty()) {
          e = ctx->pool.back();
          ctx->pool.pop_back();
        } else {
          cudaEventCreate(&e);
        }
        return e;
      };
      r.a = take();
      r.b = take();
      SGN_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(st->gexec, c.a, r.a));
      SGN_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(st->gexec, c.b, r.b));
      ctx->recs.push_back(r);
    }
  }
  SGN_CUDA(ctx, cudaEventRecord(st->ge0, s));
  SGN_CUDA(ctx, cudaStreamWaitEvent(st->gs, st->ge0, 0));
  SGN_CUDA(ctx, cudaGraphLaunch(st->gexec, st->gs));
  SGN_CUDA(ctx, cudaEventRecord(st->ge1, st->gs));
  SGN_CUDA(ctx, cudaStreamWaitEvent(s, st->ge1, 0));
  st->t += st->dt_last[0];
  st->step += 1;
  return SGN_OK;
}

// A 1d RK4 step: the first with given options runs directly; later ones replay a graph of it
// (one launch instead of ~200 launches and event operations per step).
sgn_status rk4_step(sgn_state* st, const sgn_opts* o, cudaStream_t s) {
  sgn_ctx* ctx = st->lay->ctx;
  if (st->lay->dim != 1 || st->gdisabled) return rk4_once(st, o, s);
  const bool same = st->gkey_prof == ctx->prof && st->gkey_gen == st->lay->l1.gen &&
                    same_opts(st->gkey, *o);
  if (!same) {
    graph_drop(st);
    st->gkey = *o;
    st->gkey_prof = ctx->prof;
    st->gkey_gen = st->lay->l1.gen;
    return rk4_once(st, o, s);
  }
  if (!st->gexec && graph_capture(st, o) != SGN_OK) {
    st->gdisabled = true;           // e.g. the caller is itself capturing: launch directly
    return rk4_once(st, o, s);
  }
  return graph_replay(st, s);
}

}  // namespace

extern "C" sgn_status sgn_step_rk4(sgn_state* st, const double* dt, int nsteps,
                                   const sgn_opts* opts, sgn_stream stream) {
  if (!st || !dt || nsteps < 0) return SGN_ERR_INVALID_ARG;
  DeviceGuard g(st->lay->device);
  cudaStream_t s = as_stream(stream);
  SGN_TRY(check_opts(st, opts));
  SGN_TRY(upload_dt(st, dt, s));
  st->last = s;
  for (int k = 0; k < nsteps; ++k) SGN_TRY(rk4_step(st, opts, s));
  st->hist = HIST_NONE;
  st->levels = 0;
  return SGN_OK;
}

// Adams-Bashforth (Eq:AB, Table 1): w_{n+s} = w_{n+s-1} + dt sum_j b_j f_{n+j}
extern "C" sgn_status sgn_step_abk(sgn_state* st, int order, const double* dt, int nsteps,
                                   const sgn_opts* opts, sgn_stream stream) {
  static const double B[5][4] = {{0, 0, 0, 0},
                                 {0, 0, 0, 0},
                                 {-0.5, 1.5, 0, 0},
                                 {5.0 / 12, -16.0 / 12, 23.0 / 12, 0},
                                 {-9.0 / 24, 37.0 / 24, -59.0 / 24, 55.0 / 24}};
  if (!st || !dt || nsteps < 0 || order < 2 || order > 4) return SGN_ERR_INVALID_ARG;
  DeviceGuard g(st->lay->device);
  cudaStream_t s = as_stream(stream);
  SGN_TRY(check_opts(st, opts));
  const bool same_dt = (int)st->dt_last.size() == st->lay->count &&
                       std::equal(st->dt_last.begin(), st->dt_last.end(), dt);
  if (st->hist != HIST_AB || !same_dt) st->levels = 0;
  SGN_TRY(upload_dt(st, dt, s));
  st->last = s;
  const int d = st->d;
  auto make_room = [&]() {
    // rotate so that he[levels-1] is the newest
    if (st->levels == 4) {
      std::rotate(st->he, st->he + 1, st->he + 4);
      std::rotate(st->hU, st->hU + 1, st->hU + 4);
      st->levels = 3;
    }
  };
  auto push = [&]() -> sgn_status {
    make_room();
    SGN_TRY(rhs_at(st, st->eta, st->u, st->he[st->levels], st->hU[st->levels], s));
    st->levels += 1;
    return SGN_OK;
  };
  if (st->levels == 0) SGN_TRY(push());
  st->hist = HIST_AB;
  for (int k = 0; k < nsteps; ++k) {
    if (st->levels < order) {
      SGN_TRY(rk4_once(st, opts, s));
    } else {
      const int L0 = st->levels - order;   // oldest level used
      const double* const* he = st->he + L0;
      const double* const* hU = st->hU + L0;
      if (order == 2) {
        SGN_TRY(lincomb(st, st->eta, {{st->eta, 1.0}}, {{he[0], B[2][0]}, {he[1], B[2][1]}}, 1, s,
                        st->U, {{st->U, 1.0}}, {{hU[0], B[2][0]}, {hU[1], B[2][1]}}, d));
      } else if (order == 3) {
        SGN_TRY(lincomb(st, st->eta, {{st->eta, 1.0}},
                        {{he[0], B[3][0]}, {he[1], B[3][1]}, {he[2], B[3][2]}}, 1, s, st->U,
                        {{st->U, 1.0}}, {{hU[0], B[3][0]}, {hU[1], B[3][1]}, {hU[2], B[3][2]}},
                        d));
      } else {
        SGN_TRY(lincomb(st, st->eta, {{st->eta, 1.0}},
                        {{he[0], B[4][0]}, {he[1], B[4][1]}, {he[2], B[4][2]}, {he[3], B[4][3]}},
                        1, s, st->U, {{st->U, 1.0}},
                        {{hU[0], B[4][0]}, {hU[1], B[4][1]}, {hU[2], B[4][2]}, {hU[3], B[4][3]}},
                        d));
      }
      SGN_TRY(dealias_at(st, st->eta, st->U, nullptr, s));
      // the solve for u_{n+1} and the newest history level f(w_{n+1}) (the combinations
      // above were launched with the current history pointers, so rotating is safe)
      make_room();
      SGN_TRY(advance_time(st, s));          // the new level's right-hand side is at t_{n+1}
      // the solve starts from u extrapolated from the last step (reading R8)
      const long long V = (long long)d * st->P;
      SGN_TRY(step_guess(st, 1.0, st->u_s, s));
      SGN_TRY(copy_field(st, st->u_prev, st->u, V, s));
      SGN_TRY(copy_field(st, st->u, st->u_s, V, s));
      SGN_TRY(stage_at(st, st->eta, st->U, st->u, st->he[st->levels], st->hU[st->levels], opts,
                       s, 0.0));
      SGN_TRY(copy_field(st, st->u_last, st->u, V, s));
      st->levels += 1;
      st->t += st->dt_last[0];
      st->step += 1;
      continue;
    }
    SGN_TRY(push());
  }
  return SGN_OK;
}

// Linearly implicit SBDF2 (Eq:MM):
//   w_{n+2} = (4 w_{n+1} - w_n + 2 dt (2 f_{n+1} - f_n)) / 3
//   u_{n+2} = A^{-1} [2 res_{n+1} - res_n],  res_j = A u_j - G_j u_j + U_j
extern "C" sgn_status sgn_step_linimp(sgn_state* st, const double* dt, int nsteps,
                                      const sgn_opts* opts, sgn_stream stream) {
  if (!st || !dt || nsteps < 0) return SGN_ERR_INVALID_ARG;
  sgn_ctx* ctx = st->lay->ctx;
  if (has_generic(st->lay))
    return fail(ctx, SGN_ERR_UNSUPPORTED_SIZE, "SBDF2 takes power-of-two sizes");
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  SGN_TRY(check_opts(st, opts));
  const bool same_dt = (int)st->dt_last.size() == st->lay->count &&
                       std::equal(st->dt_last.begin(), st->dt_last.end(), dt);
  if (st->hist != HIST_SBDF2 || !same_dt) st->levels = 0;
  SGN_TRY(upload_dt(st, dt, s));
  st->last = s;
  const int d = st->d;
  const long long P = st->P, V = d * P;
  const bool one_d = st->lay->dim == 1;
  // 1d: the residual and the A-solve run as one launch (transforms in double-float on the
  // mixed path) that writes the new u into u_s and hands u_x to the right-hand side of the
  // same level; 2d: residual and solve launches.
  auto res_of = [&](const double* eta, const double* u, const double* U, void* out) -> sgn_status {
    cudaError_t e =
        one_d ? sgn::launch_linimp_step1d(st->lay->l1, ctx->tw64, ctx->tw32, st->prec,
                                          st->A_fixed, eta, st->gradh, const_cast<double*>(u),
                                          U, nullptr, out, 0.0, 0.0, false, st->lay->ws,
                                          nullptr, nullptr, s)
              : sgn::launch_linimp_res2d(st->lay->l2, ctx->tw64, st->A_fixed, eta, st->gradh, u,
                                         U, out, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "linimp residual");
    return SGN_OK;
  };
  for (int k = 0; k < nsteps; ++k) {
    if (st->levels == 0) {
      // start-up: keep level n, take one RK4 step to level n+1
      SGN_TRY(copy_field(st, st->eta_p, st->eta, P, s));
      SGN_TRY(copy_field(st, st->U_p, st->U, V, s));
      SGN_TRY(rhs_at(st, st->eta, st->u, st->he[0], st->hU[0], s));
      SGN_TRY(res_of(st->eta, st->u, st->U, st->res0));
      SGN_TRY(rk4_once(st, opts, s));
      st->levels = 2;
      st->hist = HIST_SBDF2;
      continue;
    }
    // res_{n+1} into res1 and (1d) u_{n+2} into u_s with u_x handed over, then f_{n+1} into
    // he[1] from the same level (2d: f_{n+1}, then the residual)
    if (one_d) {
      sgn_layout* lay = st->lay;
      cudaError_t e = sgn::launch_linimp_step1d(lay->l1, ctx->tw64, ctx->tw32, st->prec,
                                                st->A_fixed, st->eta, st->gradh, st->u, st->U,
                                                st->res0, st->res1, 2.0, -1.0, true, lay->ws,
                                                st->u_s, lay->scratch, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "linimp step");
      {
        ProfScope prof(ctx, s, 1);
        e = sgn::launch_rhs1d_ux(lay->l1, ctx->tw64, ctx->tw32, st->prec, lay->grids[0].g,
                                 st->eta, st->u, st->h, st->gradh, st->he[1], st->hU[1],
                                 lay->scratch, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rhs launch");
      }
      SGN_TRY(force_at(st, st->he[1], st->hU[1], 0.0, s));
    } else {
      SGN_TRY(rhs_at(st, st->eta, st->u, st->he[1], st->hU[1], s));
      SGN_TRY(res_of(st->eta, st->u, st->U, st->res1));
    }
    SGN_TRY(lincomb(st, st->eta_s, {{st->eta, 4.0 / 3.0}, {st->eta_p, -1.0 / 3.0}},
                    {{st->he[1], 4.0 / 3.0}, {st->he[0], -2.0 / 3.0}}, 1, s, st->U_s,
                    {{st->U, 4.0 / 3.0}, {st->U_p, -1.0 / 3.0}},
                    {{st->hU[1], 4.0 / 3.0}, {st->hU[0], -2.0 / 3.0}}, d));
    if (!one_d) {
      cudaError_t e = sgn::launch_linimp_solve2d(st->lay->l2, ctx->tw64, st->A_fixed, st->res1,
                                                 st->res0, 2.0, -1.0, st->u_s, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "linimp solve");
    }
    SGN_TRY(copy_field(st, st->u, st->u_s, V, s));
    SGN_TRY(copy_field(st, st->eta_p, st->eta, P, s));
    SGN_TRY(copy_field(st, st->U_p, st->U, V, s));
    SGN_TRY(copy_field(st, st->eta, st->eta_s, P, s));
    SGN_TRY(copy_field(st, st->U, st->U_s, V, s));
    SGN_TRY(dealias_at(st, st->eta, st->U, st->u, s));
    if (one_d) {
      k_sbdf2_guard<<<st->lay->count, 256, 0, s>>>(st->lay->l1.d_inst, st->P, st->eta,
                                                   st->A_fixed, st->stats);
    } else {
      const long long nb = std::min<long long>(1024, (st->P + 255) / 256);
      k_sbdf2_guard2d<<<(int)nb, 256, 0, s>>>(st->P, st->eta, st->A_fixed, st->stats);
    }
    SGN_CUDA(ctx, cudaGetLastError());
    std::swap(st->he[0], st->he[1]);
    std::swap(st->hU[0], st->hU[1]);
    std::swap(st->res0, st->res1);
    SGN_TRY(advance_time(st, s));
    st->t += st->dt_last[0];
    st->step += 1;
  }
  return SGN_OK;
}

namespace {

// One RK4 step of the non-constraint form on (eta, u): stage i takes (f_eta, u_t) with
// G_{eta_i,h} u_t = M(eta_i, u_i) (warm start from the previous u_t); u_t stages live in hU[]
// (the multistep history is reset), M in fU[].  U = G u afterwards.
sgn_status rk4_nc_once(sgn_state* st, const sgn_opts* o, cudaStream_t s) {
  sgn_layout* lay = st->lay;
  sgn_ctx* ctx = lay->ctx;
  const int d = st->d;
  const long long V = (long long)d * st->P;
  const bool one_d = lay->dim == 1;
  static const double a[4] = {0.0, 0.5, 0.5, 1.0};
  for (int i = 0; i < 4; ++i) {
    const double* eta_i = st->eta;
    const double* u_i = st->u;
    if (i > 0) {
      SGN_TRY(lincomb(st, st->eta_s, {{st->eta, 1.0}}, {{st->fe[i - 1], a[i]}}, 1, s, st->u_s,
                      {{st->u, 1.0}}, {{st->hU[i - 1], a[i]}}, d));
      eta_i = st->eta_s;
      u_i = st->u_s;
    }
    {
      ProfScope prof(ctx, s, 1);
      const cudaError_t e =
          one_d ? sgn::launch_rhs_nc1d(lay->l1, ctx->tw64, ctx->tw32, o->prec, lay->grids[0].g,
                                       eta_i, u_i, st->h, st->gradh, st->fe[i], st->fU[i],
                                       lay->scratch, s)
                : sgn::launch_rhs_nc2d(lay->l2, ctx->tw64, lay->grids[0].g, eta_i, u_i, st->h,
                                       st->gradh, st->fe[i], st->fU[i], s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "non-constraint rhs launch");
    }
    // warm start: the previous u_t; stage 4 (c = 1) from 2 u_t^(3) - u_t^(1) (c = 1/2, 0)
    if (i == 3)
      SGN_TRY(lincomb(st, st->hU[3], {{st->hU[2], 2.0}, {st->hU[0], -1.0}}, {}, d, s));
    else
      SGN_TRY(copy_field(st, st->hU[i], i == 0 ? st->ut : st->hU[i - 1], V, s));
    SGN_TRY(solve_at(st, eta_i, st->fU[i], st->hU[i], o, s));
  }
  const double b0 = 1.0 / 6.0, b1 = 1.0 / 3.0;
  SGN_TRY(lincomb(st, st->eta, {{st->eta, 1.0}},
                  {{st->fe[0], b0}, {st->fe[1], b1}, {st->fe[2], b1}, {st->fe[3], b0}}, 1, s,
                  st->u, {{st->u, 1.0}},
                  {{st->hU[0], b0}, {st->hU[1], b1}, {st->hU[2], b1}, {st->hU[3], b0}}, d));
  const cudaError_t e =
      one_d ? sgn::launch_apply_G1d(lay->l1, ctx->tw64, st->eta, st->gradh, st->u, st->U, s)
            : sgn::launch_apply_G2d(lay->l2, ctx->tw64, st->eta, st->gradh, st->u, st->U, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "apply G");
  SGN_TRY(copy_field(st, st->ut, st->hU[3], V, s));
  SGN_TRY(advance_time(st, s));
  st->t += st->dt_last[0];
  st->step += 1;
  return SGN_OK;
}

}  // namespace

extern "C" sgn_status sgn_step_rk4_nc(sgn_state* st, const double* dt, int nsteps,
                                      const sgn_opts* opts, sgn_stream stream) {
  if (!st || !dt || nsteps < 0) return SGN_ERR_INVALID_ARG;
  if (has_generic(st->lay))
    return fail(st->lay->ctx, SGN_ERR_UNSUPPORTED_SIZE,
                "the non-constraint stepper takes power-of-two sizes");
  if (st->force.K > 0 || st->dealias)
    return fail(st->lay->ctx, SGN_ERR_INVALID_ARG,
                "the non-constraint stepper takes states without forcing or dealiasing");
  DeviceGuard g(st->lay->device);
  cudaStream_t s = as_stream(stream);
  SGN_TRY(check_opts(st, opts));
  SGN_TRY(upload_dt(st, dt, s));
  st->last = s;
  st->hist = HIST_NONE;                  // hU[] holds u_t stages here
  st->levels = 0;
  for (int k = 0; k < nsteps; ++k) SGN_TRY(rk4_nc_once(st, opts, s));
  return SGN_OK;
}

extern "C" sgn_status sgn_state_set_forcing(sgn_state* st, int nterms, const double* phi_eta,
                                            const double* phi_U, const double* omega,
                                            const double* theta) {
  if (!st || nterms < 0 || nterms > SGN_MAX_FORCING ||
      (nterms > 0 && (!phi_eta || !phi_U || !omega || !theta)))
    return SGN_ERR_INVALID_ARG;
  for (int k = 0; k < nterms; ++k)
    if (!std::isfinite(omega[k]) || !std::isfinite(theta[k])) return SGN_ERR_INVALID_ARG;
  DeviceGuard g(st->lay->device);
  ForceTerms F{};
  F.K = nterms;
  for (int k = 0; k < nterms; ++k) {
    F.pe[k] = phi_eta + (long long)k * st->P;
    F.pu[k] = phi_U + (long long)k * st->d * st->P;
    F.omega[k] = omega[k];
    F.theta[k] = theta[k];
  }
  st->force = F;
  graph_drop(st);                   // a captured step holds the previous terms
  return SGN_OK;
}


extern "C" sgn_status sgn_state_set_dealias(sgn_state* st, int on) {
  if (!st) return SGN_ERR_INVALID_ARG;
  if (on && has_generic(st->lay))
    return fail(st->lay->ctx, SGN_ERR_UNSUPPORTED_SIZE, "dealiasing takes power-of-two sizes");
  st->dealias = on ? 1 : 0;
  graph_drop(st);                   // a captured step holds the previous setting
  return SGN_OK;
}

namespace {

// The autotuner of a 2d state: the inner-solve form of its layout (the persistent launch
// or four kernels per inner iteration), each timed on RK4 steps of the state's own problem
// from the same saved state, in two passes; the persistent form stays unless the other is
// at least 3% faster.  The state is restored afterwards.
sgn_status autotune_2d(sgn_state* st, const sgn_opts* opts, cudaStream_t s, double* best_ms) {
  sgn_layout* lay = st->lay;
  sgn_ctx* ctx = lay->ctx;
  sgn::Layout2d& L = lay->l2;
  const long long P = st->P, V = 2 * P;
  double* save = nullptr;
  if (cudaMalloc(&save, sizeof(double) * (P + 2 * V + 1) + sizeof(DevStats)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SGN_ERR_NOMEM, "autotune buffers");
  }
  DevStats* save_stats = reinterpret_cast<DevStats*>(save + P + 2 * V + 1);
  const double t0 = st->t;
  const long long k0 = st->step;
  auto copy_state = [&](bool to_save) -> sgn_status {
    double* f[3] = {st->eta, st->U, st->u};
    const long long len[3] = {P, V, V}, at[3] = {0, P, P + V};
    for (int i = 0; i < 3; ++i)
      SGN_CUDA(ctx, cudaMemcpyAsync(to_save ? save + at[i] : f[i], to_save ? f[i] : save + at[i],
                                    sizeof(double) * len[i], cudaMemcpyDeviceToDevice, s));
    SGN_CUDA(ctx, cudaMemcpyAsync(to_save ? save + P + 2 * V : st->t_dev,
                                  to_save ? st->t_dev : save + P + 2 * V, sizeof(double),
                                  cudaMemcpyDeviceToDevice, s));
    SGN_CUDA(ctx, cudaMemcpyAsync(to_save ? (void*)save_stats : (void*)st->stats,
                                  to_save ? (const void*)st->stats : (const void*)save_stats,
                                  sizeof(DevStats), cudaMemcpyDeviceToDevice, s));
    st->t = t0;
    st->step = k0;
    return SGN_OK;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sgn_status r = copy_state(true);
  if (!r && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    cudaGetLastError();
    r = fail(ctx, SGN_ERR_CUDA, "autotune events");
  }
  constexpr int kTimed = 2;
  // candidates: the persistent form with radix-8 stages and units sized by their count (the
  // default), the same with 128 and with 256 threads per unit, with radix-16 stages, and the
  // four-kernel form
  constexpr int kCand = 5;
  const int cform[kCand] = {0, 0, 0, 0, 1}, cmaxb[kCand] = {3, 3, 3, 4, 3};
  const int cgt[kCand] = {0, 128, 256, 0, 0};
  float t_of[kCand] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const int tw = L.p_tw;
  for (int pass = 0; pass < 2 && !r; ++pass) {
    for (int c = 0; c < kCand && !r; ++c) {
      if (sgn::layout2d_set_inner_form(L, cform[c], tw) != cudaSuccess ||
          sgn::layout2d_set_radix(L, cmaxb[c]) != cudaSuccess ||
          sgn::layout2d_set_unit_threads(L, cgt[c]) != cudaSuccess)
        r = cuda_fail(ctx, cudaGetLastError(), "autotune form");
      if (!r) r = rk4_step(st, opts, s);              // untimed: builds the solve graph
      if (!r) r = copy_state(false);
      if (!r && cudaEventRecord(e0, s) != cudaSuccess)
        r = cuda_fail(ctx, cudaGetLastError(), "autotune");
      for (int k = 0; k < kTimed && !r; ++k) r = rk4_step(st, opts, s);
      float ms = 0.0f;
      if (!r && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        r = cuda_fail(ctx, cudaGetLastError(), "autotune timing");
      if (!r) r = copy_state(false);
      if (!r && (pass == 0 || ms < t_of[c])) t_of[c] = ms;
    }
  }
  int best = 0;
  for (int c = 1; c < kCand; ++c)
    if (t_of[c] < 0.97f * t_of[0] && t_of[c] < t_of[best]) best = c;
  sgn::layout2d_set_inner_form(L, cform[best], tw);
  sgn::layout2d_set_radix(L, cmaxb[best]);
  sgn::layout2d_set_unit_threads(L, cgt[best]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the state is as it was before tuning, with no RK4 history (as after sgn_state_init)
  cudaMemsetAsync(st->u_last, 0xff, sizeof(double) * st->d * st->P, s);
  cudaStreamSynchronize(s);
  cudaFree(save);
  st->last = s;
  if (r) return r;
  if (best_ms) *best_ms = t_of[best] / kTimed;
  return SGN_OK;
}

}  // namespace

extern "C" sgn_status sgn_state_autotune(sgn_state* st, const double* dt, const sgn_opts* opts,
                                         sgn_stream stream, double* best_ms) {
  if (!st || !dt || !opts) return SGN_ERR_INVALID_ARG;
  if (best_ms) *best_ms = 0.0;
  sgn_layout* lay = st->lay;
  if (lay->dim == 2) {
    DeviceGuard g(lay->ctx->device);
    cudaStream_t s = as_stream(stream);
    SGN_TRY(check_opts(st, opts));
    SGN_TRY(upload_dt(st, dt, s));
    if (lay->l2.mr) return SGN_OK;                 // one form: nothing to choose
    return autotune_2d(st, opts, s, best_ms);
  }
  sgn_ctx* ctx = lay->ctx;
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(stream);
  sgn::Layout1d& L = lay->l1;
  std::vector<int> cls;                              // classes with a choice of form
  for (int l = sgn::kClusterLog1d; l <= sgn::kSmemLog1d; ++l)
    if (L.class_end[l] > L.class_begin[l]) cls.push_back(l);
  if (cls.empty()) return SGN_OK;
  SGN_TRY(check_opts(st, opts));
  SGN_TRY(upload_dt(st, dt, s));
  // the state to come back to before every timing and at the end
  const long long P = st->P;
  double* save = nullptr;
  if (cudaMalloc(&save, sizeof(double) * (3 * (size_t)P + L.count) + sizeof(DevStats)) !=
      cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SGN_ERR_NOMEM, "autotune buffers");
  }
  DevStats* save_stats = reinterpret_cast<DevStats*>(save + 3 * P + L.count);
  const double t0 = st->t;
  const long long k0 = st->step;
  auto copy3 = [&](bool to_save) -> sgn_status {
    double* f[3] = {st->eta, st->U, st->u};
    for (int i = 0; i < 3; ++i) {
      double* src = to_save ? f[i] : save + i * P;
      double* dst = to_save ? save + i * P : f[i];
      SGN_CUDA(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
    }
    SGN_CUDA(ctx, cudaMemcpyAsync(to_save ? save + 3 * P : st->t_dev,
                                  to_save ? st->t_dev : save + 3 * P,
                                  sizeof(double) * L.count, cudaMemcpyDeviceToDevice, s));
    SGN_CUDA(ctx, cudaMemcpyAsync(to_save ? (void*)save_stats : (void*)st->stats,
                                  to_save ? (const void*)st->stats : (const void*)save_stats,
                                  sizeof(DevStats), cudaMemcpyDeviceToDevice, s));
    st->t = t0;
    st->step = k0;
    return SGN_OK;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sgn_status r = copy3(true);
  if (!r && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    cudaGetLastError();
    r = fail(ctx, SGN_ERR_CUDA, "autotune events");
  }
  // every combination of forms over the classes (solve and right-hand side separately),
  // from the same state: one untimed RK4 step (loads the kernels), then two timed (direct
  // launches: no graph capture in the timing)
  auto apply = [&](int c) {
    for (size_t i = 0; i < cls.size(); ++i) {
      L.form[cls[i]] = (c >> (2 * i)) & 1 ? 2 : 1;
      L.rform[cls[i]] = (c >> (2 * i + 1)) & 1 ? 2 : 1;
    }
  };
  // Each combination is timed as steps run in production: its own captured step graph
  // (two untimed steps: direct launches, then capture), then three timed replays, in two
  // passes over all combinations, keeping each one's faster pass.  (Timed on direct
  // launches, two-CTA forms for n = 8192 looked 3% faster and replayed 5% slower.)  A
  // combination other than the default (one CTA everywhere) is taken only when it is at
  // least 3% faster: a winner within the timing noise of a few steps would be a coin toss.
  const int combos = 1 << (2 * (int)cls.size());
  constexpr int kTimed = 3;
  std::vector<float> t_of(combos, 0.0f);
  for (int pass = 0; pass < 2 && !r; ++pass) {
    for (int c = 0; c < combos && !r; ++c) {
      apply(c);
      L.gen += 1;                                  // a new graph key: capture this form
      for (int k = 0; k < 2 && !r; ++k) r = rk4_step(st, opts, s);
      if (!r) r = copy3(false);
      if (!r && cudaEventRecord(e0, s) != cudaSuccess)
        r = cuda_fail(ctx, cudaGetLastError(), "autotune");
      for (int k = 0; k < kTimed && !r; ++k) r = rk4_step(st, opts, s);
      float ms = 0.0f;
      if (!r && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        r = cuda_fail(ctx, cudaGetLastError(), "autotune timing");
      if (!r) r = copy3(false);
      if (!r && (pass == 0 || ms < t_of[c])) t_of[c] = ms;
    }
  }
  int best = 0;
  for (int c = 1; c < combos; ++c)
    if (t_of[c] < 0.97f * t_of[0] && t_of[c] < t_of[best]) best = c;
  const float best_t = t_of[best];
  apply(best);
  L.gen += 1;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the state is as it was before tuning, with no RK4 history (as after sgn_state_init)
  cudaMemsetAsync(st->u_last, 0xff, sizeof(double) * st->d * st->P, s);
  cudaStreamSynchronize(s);
  cudaFree(save);
  st->last = s;
  if (r) return r;
  if (best_ms) *best_ms = best_t / kTimed;
  return SGN_OK;
}

extern "C" sgn_status sgn_state_get_stats(sgn_state* st, sgn_state_stats* out) {
  if (!st || !out) return SGN_ERR_INVALID_ARG;
  sgn_ctx* ctx = st->lay->ctx;
  DeviceGuard g(ctx->device);
  DevStats h{};
  SGN_CUDA(ctx, cudaMemcpyAsync(&h, st->stats, sizeof(DevStats), cudaMemcpyDeviceToHost, st->last));
  SGN_CUDA(ctx, cudaStreamSynchronize(st->last));
  out->solves = h.solves;
  out->iterations = h.iterations;
  out->max_iters = h.max_iters;
  out->status = h.status;
  out->t = st->t;
  out->step = st->step;
  out->flops32 = h.flops32;
  out->flops64 = h.flops64;
  out->refinements = h.refinements;
  out->sbdf2_stability_warnings = h.sbdf2_warn;
  return SGN_OK;
}

extern "C" void sgn_state_free(sgn_state* st) {
  if (!st) return;
  DeviceGuard g(st->lay->device);
  graph_drop(st);
  if (st->gs) cudaStreamDestroy(st->gs);
  if (st->ge0) cudaEventDestroy(st->ge0);
  if (st->ge1) cudaEventDestroy(st->ge1);
  for (double* p : st->bufs) cudaFree(p);
  cudaFree(st->res0);
  cudaFree(st->res1);
  cudaFree(st->A_fixed);
  cudaFree(st->stats);
  delete st;
}
