// Allocation-free entry point: the 1d constraint solve of sgn_pcg for one instance, with
// every buffer it needs held in file-scope static device arrays instead of memory from
// cudaMalloc.  It exists for callers that cannot allocate device memory at solve time:
// code running under an allocator that forbids new allocations once a run has started
// (a pre-reserved memory pool, an embedded or safety-certified host that freezes the heap
// after start-up), or a host library that must not trigger the CUDA allocator from inside
// a time-step callback.
//
// Nothing here changes the other entry points; it reuses the same kernel launcher.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/sgn.h"
#include "sgn_internal.h"

namespace {

constexpr long long kWsCplx = (long long)sgn::kWsVectors * (SGN_NOALLOC_MAX_N / 2 + 1);

// The scratch of the solve (six half spectra of n/2 + 1 complex doubles), the twiddle
// tables, the instance descriptor and the solve record.  Every GPU that loads this library
// holds these arrays (about 1 MB) until the process exits.
static __device__ __align__(256) double g_ws[2 * kWsCplx];
static __device__ __align__(256) double g_tw64[2 * sgn::kTwiddleN];
static __device__ __align__(256) float g_tw32[(sgn::kTw32Bytes + sgn::kTwDfBytes) / sizeof(float)];
static __device__ __align__(256) float g_coef_df[6 * SGN_NOALLOC_MAX_N];
static __device__ __align__(256) sgn::Inst1d g_inst[1];
static __device__ __align__(256) int g_ids[1];
static __device__ __align__(256) sgn::SolveRec g_rec[1];

// Host-side device addresses of the arrays above.  In host code the array names are host
// stand-ins, not device addresses, so the kernels get these looked-up pointers.
struct DevicePtrs {
  bool ready = false;
  void* ws = nullptr;
  void* tw64 = nullptr;
  void* tw32 = nullptr;
  sgn::Inst1d* inst = nullptr;
  int* ids = nullptr;
  sgn::SolveRec* rec = nullptr;
  float* coef_df = nullptr;
};

// Writes this call's instance descriptor (from launch arguments, so nothing is read from
// host memory) and the constant instance index, and clears the solve record so that a
// failed launch cannot report the previous call's result.
__global__ void k_noalloc_prepare(sgn::Inst1d* inst, int* ids, sgn::SolveRec* rec, int n,
                                  int log2n, double L) {
  inst->n = n;
  inst->log2n = log2n;
  inst->L = L;
  inst->off = 0;
  inst->ws = 0;
  inst->tw = 0;
  inst->gbuf = -1;
  ids[0] = 0;
  *rec = sgn::SolveRec{};
}

constexpr int kMaxDevices = 64;
DevicePtrs g_ptrs[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: look up the symbol addresses and fill the
// twiddle tables, then wait for that work.  Under CUDA's lazy module loading the first
// lookup is also where the driver loads this module and places its static arrays.
sgn_status setup_device(int dev, cudaStream_t s) {
  DevicePtrs& P = g_ptrs[dev];
  if (P.ready) return SGN_OK;
  if (cudaGetSymbolAddress(&P.ws, g_ws) != cudaSuccess ||
      cudaGetSymbolAddress(&P.tw64, g_tw64) != cudaSuccess ||
      cudaGetSymbolAddress(&P.tw32, g_tw32) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&P.inst), g_inst) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&P.ids), g_ids) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&P.rec), g_rec) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&P.coef_df), g_coef_df) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  if (sgn::twiddles_init(P.tw64, P.tw32, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  P.ready = true;
  return SGN_OK;
}

}  // namespace

extern "C" sgn_status sgn_pcg1d_noalloc(int n, double L, const double* eta, const double* gradh,
                                        const double* b, double* x, double rtol, int maxit,
                                        sgn_precision prec, sgn_pcg_info* info,
                                        sgn_stream stream) {
  int log2n = -1;
  for (int l = 3; l <= 13; ++l)
    if (n == (1 << l)) log2n = l;
  if (n > SGN_NOALLOC_MAX_N || log2n < 0) return SGN_ERR_UNSUPPORTED_SIZE;
  if (!eta || !gradh || !b || !x || !(L > 0.0) || !(rtol > 0.0) || maxit < 0 ||
      (prec != SGN_PREC_FP64 && prec != SGN_PREC_MIXED))
    return SGN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  DevicePtrs P;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    sgn_status st = setup_device(dev, s);
    if (st != SGN_OK) return st;
    P = g_ptrs[dev];
  }
  k_noalloc_prepare<<<1, 1, 0, s>>>(P.inst, P.ids, P.rec, n, log2n, L);
  if (cudaGetLastError() != cudaSuccess) return SGN_ERR_CUDA;
  sgn::Layout1d lay;
  lay.count = 1;
  lay.points = n;
  lay.ws_cplx = (long long)sgn::kWsVectors * (n / 2 + 1);
  lay.d_inst = P.inst;
  lay.d_ids = P.ids;
  lay.class_begin[log2n] = 0;
  lay.class_end[log2n] = 1;
  cudaError_t e = sgn::launch_pcg1d(lay, P.tw64, P.tw32, prec, eta, gradh, b, x, nullptr,
                                    SGN_COEF_OPT, rtol, -1.0, maxit, 12, P.rec, P.ws,
                                    P.coef_df, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  if (!info) return SGN_OK;
  sgn::SolveRec R;
  if (cudaMemcpyAsync(&R, P.rec, sizeof(R), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  info->iters = R.iters;
  info->refinements = R.refinements;
  info->rel_resid_Ainv = R.ratio;
  info->status = R.status;
  return R.status == SGN_OK ? SGN_OK : (sgn_status)R.status;
}
