// Device helpers shared by the 2d kernel translation units (sgn_2d.cu, sgn_2d_pcg.cu):
// the device-resident scalars of a solve, wavenumbers, the per-mode A^{-1}, twiddle
// tables per precision, and the packed real-row transforms of the row passes.
#pragma once
#include <type_traits>

#include "sgn_1d_dev.cuh"
#include "sgn_2d.h"

namespace sgn {

// device-resident scalars of one 2d solve
struct Scal2d {
  double bb;           // b.A^{-1}b (high precision problem)
  double rz;           // inner r.z
  double rz64;         // refinement residual r.A^{-1}r
  double alpha, beta;
  double tol;          // inner absolute tolerance on sqrt(r.z)
  int done;            // inner loop finished
  int iters;           // inner iterations (this solve)
  int cap;             // iteration cap
  int status;
  unsigned int ticket; // last-block counter
  double sigma, alpha_A, kappa_ub, eta_min, eta_max;
  int flat;
  // float32 copies for the inner solve's kernels, written where the doubles are: on this
  // part a float64 instruction costs 62 float32 ones, so per-mode work stays in float32
  float sigf, alphaAf, isigf;   // sigma, alpha of A and 1 / sigma
  float alphaf, betaf;          // CG alpha, beta
  // device-driven solve (the cached solve graph): options, and the refinement loop's state
  double rtol, rtol_in;         // outer tolerance; inner tolerance (<= 0: adaptive)
  double rn;                    // ||r||_{A^{-1}} of the last refinement residual
  int maxit, max_refine, kind;
  int refinements, it_before;
};

namespace d2 {

using d1::kPi;
using d1::kLambdaPlus;
using d1::kLambdaMinus;
using d1::kFlatSlope;

constexpr int kRowNT = 256;
constexpr int kColNT = 512;
constexpr int kMaxParts = 2048;

// ---- mode helpers --------------------------------------------------------------------
struct Modes2d {
  int nx, ny, H;
  double kxu, kyu;     // 2 pi / Lx, 2 pi / Ly
  __device__ __forceinline__ double kx(int c) const { return c == (nx >> 1) ? 0.0 : kxu * c; }
  __device__ __forceinline__ double ky(int y) const { return kyu * wave_index(y, ny); }
  __device__ __forceinline__ double weight(int c) const {
    return (c == 0 || c == (nx >> 1)) ? 1.0 : 2.0;
  }
};

inline Modes2d modes_of(const Layout2d& L) {
  Modes2d M;
  M.nx = L.nx;
  M.ny = L.ny;
  M.H = L.nx / 2 + 1;
  M.kxu = 2.0 * kPi / L.Lx;
  M.kyu = 2.0 * kPi / L.Ly;
  return M;
}

template <typename T>
__device__ __forceinline__ cplx<T> mul_ik(cplx<T> a, T k) {   // i k a
  return mk(-(a.y * k), a.x * k);
}

template <typename T>
__device__ __forceinline__ cplx<T> ld_c(const void* base, long long i) {
  return reinterpret_cast<const cplx<T>*>(base)[i];
}
template <typename T>
__device__ __forceinline__ void st_c(void* base, long long i, cplx<T> v) {
  reinterpret_cast<cplx<T>*>(base)[i] = v;
}

// the twiddle table of each precision
template <typename T>
struct Tw;
template <>
struct Tw<double> {
  static __device__ __forceinline__ const cplx<double>* get(const void* t64, const void* t32) {
    return static_cast<const cplx<double>*>(t64);
  }
};
template <>
struct Tw<float> {
  static __device__ __forceinline__ const cplx<float>* get(const void* t64, const void* t32) {
    return static_cast<const cplx<float>*>(t32);
  }
};
template <>
struct Tw<df> {
  static __device__ __forceinline__ const cplx<df>* get(const void* t64, const void* t32) {
    return reinterpret_cast<const cplx<df>*>(static_cast<const char*>(t32) + kTw32Bytes);
  }
};

// ---- per-mode arithmetic in the working precision ---------------------------------------
// float32 for the float32 kernels of the inner solve, float64 otherwise.
template <typename T>
struct WorkP {
  using type = double;
};
template <>
struct WorkP<float> {
  using type = float;
};

template <typename TP>
struct ModesT {
  TP kxu, kyu;
  int nx, ny;
  __device__ __forceinline__ explicit ModesT(const Modes2d& M)
      : kxu((TP)M.kxu), kyu((TP)M.kyu), nx(M.nx), ny(M.ny) {}
  __device__ __forceinline__ TP kx(int c) const { return c == (nx >> 1) ? TP(0) : kxu * (TP)c; }
  __device__ __forceinline__ TP ky(int y) const { return kyu * (TP)wave_index(y, ny); }
  __device__ __forceinline__ TP weight(int c) const {
    return (c == 0 || c == (nx >> 1)) ? TP(1) : TP(2);
  }
};

// z = A^{-1} r per mode (Sherman-Morrison of sigma I + alpha k k^T)
template <typename TP>
struct AinvT {
  TP sigma, alpha, isig;
  __device__ __forceinline__ void apply(TP kx, TP ky, cplx<TP> r1, cplx<TP> r2, cplx<TP>& z1,
                                        cplx<TP>& z2) const {
    const TP f = alpha * recip(sigma + alpha * (kx * kx + ky * ky));
    const cplx<TP> kr = r1 * kx + r2 * ky;
    z1 = (r1 - kr * (f * kx)) * isig;
    z2 = (r2 - kr * (f * ky)) * isig;
  }
};
__device__ __forceinline__ AinvT<float> ainv_of(const Scal2d* sc, float) {
  return AinvT<float>{sc->sigf, sc->alphaAf, sc->isigf};
}
__device__ __forceinline__ AinvT<double> ainv_of(const Scal2d* sc, double) {
  return AinvT<double>{sc->sigma, sc->alpha_A, 1.0 / sc->sigma};
}
__device__ __forceinline__ float cg_alpha(const Scal2d* sc, float) { return sc->alphaf; }
__device__ __forceinline__ double cg_alpha(const Scal2d* sc, double) { return sc->alpha; }
__device__ __forceinline__ float cg_beta(const Scal2d* sc, float) { return sc->betaf; }
__device__ __forceinline__ double cg_beta(const Scal2d* sc, double) { return sc->beta; }

// 2^-e in T (exact), for the 1 / (nx ny) of the inverse transforms
template <typename T>
__device__ __forceinline__ T pow2_inv(int e) {
  const float f = __int_as_float((127 - e) << 23);
  if constexpr (std::is_same<T, df>::value) return df(f, 0.0f);
  else return (T)f;
}

// wavenumber of column c (x) or row y in the number type T of a kernel's data
template <typename T, typename TP>
__device__ __forceinline__ T mode_k(const ModesT<TP>& MT, int i, bool xdir) {
  const TP k = xdir ? MT.kx(i) : MT.ky(i);
  if constexpr (std::is_same<T, df>::value) return df((double)k);
  else return (T)k;
}

// high-precision value -> working precision, and back, without float64 where T is float
template <typename T>
__device__ __forceinline__ T to_work(double v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T to_work(df v) { return (T)to_f64(v); }
template <>
__device__ __forceinline__ float to_work<float>(df v) { return v.hi + v.lo; }
template <typename TH>
__device__ __forceinline__ TH widen(float v) { return (TH)v; }
template <>
__device__ __forceinline__ df widen<df>(float v) { return df(v, 0.0f); }
template <typename TH>
__device__ __forceinline__ TH widen(double v) { return num<TH>(v); }

// C2R of one packed pair: buf <- A + i B over the full row from two half rows, iFFT.
template <typename T>
__device__ __forceinline__ void load_c2r_pair(cplx<T>* z, const cplx<T>* A, const cplx<T>* B,
                                              int nx, int NT) {
  const int h = nx >> 1;
  for (int m = threadIdx.x; m < nx; m += NT) {
    cplx<T> a, b;
    if (m <= h) {
      a = A[m];
      b = B[m];
    } else {
      a = conj(A[nx - m]);
      b = conj(B[nx - m]);
    }
    // a + i b
    z[m] = mk(a.x - b.y, a.y + b.x);
  }
}

// R2C split of a packed FFT row Y = FFT(a + i b): A[m] = (Y_m + conj Y_{n-m})/2,
// B[m] = (Y_m - conj Y_{n-m})/(2i), m = 0..nx/2.
template <typename T>
__device__ __forceinline__ void split_r2c_pair(const cplx<T>* Y, cplx<T>* A, cplx<T>* B, int nx,
                                               int NT) {
  const int h = nx >> 1;
  for (int m = threadIdx.x; m <= h; m += NT) {
    cplx<T> y = Y[m], yc = conj(Y[(nx - m) & (nx - 1)]);
    cplx<T> s = y + yc, d = mul_mi(y - yc);
    A[m] = mk(half(s.x), half(s.y));
    B[m] = mk(half(d.x), half(d.y));
  }
}

// ---- persistent inner solve (sgn_2d_pcg.cu) --------------------------------------------
constexpr int kMaxBatch2d = kMaxBatch2dAbi;   // instances of one persistent inner solve

// One instance of a persistent float32 inner solve: half planes [ny][H] of complex float.
struct PInst2d {
  cplx<float>* x[2];      // correction
  cplx<float>* r[2];      // residual
  cplx<float>* p[2];      // search direction
  cplx<float>* t[3];      // transform planes
  const float* ehh;       // float32 eta, h_x, h_y: three planes of nx ny
  Scal2d* sc;             // tolerance, cap, A's symbol in; iterations, r.z, status out
  double kxu, kyu;        // 2 pi / Lx, 2 pi / Ly
};

struct PersistArgs2d {
  const PInst2d* inst;    // [B] (device)
  int B;
  int nx, ny, H, lognx, logny;
  int tw;                 // columns per column tile
  int maxb;               // log2 of the largest radix of the transforms' stages (3 or 4)
  int gt;                 // threads per unit: 128, 256, or 0 (chosen by the unit count)
  int col_units, row_units;    // per instance: column tiles, row pairs
  double* parts;          // B (row_units + col_units) per-unit partial sums
  unsigned* bar;          // arrival counter of the grid barriers
  int* err;               // set when a barrier wait gives up
  const void* tw32;       // float32 twiddle table
};

}  // namespace d2

// Launchers of the persistent inner solve (sgn_2d_pcg.cu).
// CTAs of the cooperative grid: every SM's resident CTAs, at most the largest phase's units
cudaError_t persist2d_grid(int nx, int ny, int B, int* grid);
// Zeroes the barrier words, then runs the inner solves of args.inst[0..B) to completion.
cudaError_t launch_pcg2d_persist(const d2::PersistArgs2d& args, int grid, cudaStream_t s);

}  // namespace sgn
