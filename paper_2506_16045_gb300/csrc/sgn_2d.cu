// 2d (doubly periodic) kernels: spectral derivatives, G-matvec, A^{-1}, PCG (float64, or
// float32 inner solves inside double-float refinement), right-hand side, SBDF2 pieces.
//
// Layout.  Real fields are [ny][nx] row-major; a vector field is two such planes.  Spectra
// of real fields are half spectra [ny][H], H = nx/2 + 1 (kx = 0..nx/2, all ky).  A 2d
// transform is a row pass (two real rows packed into one complex FFT of length nx, split
// into two half rows by Hermitian symmetry) and a column pass (tiles of TW half-spectrum
// columns transposed into shared memory and transformed as a batch of length-ny FFTs).
//
// Matvec (Def:G, §2.2, in the weak form of Def:MatrixM): with d = div p,
//   w = eta (I + grad h grad h^T) p + eta^2/2 grad h d,   q = eta^2/2 grad h . p + eta^3/3 d,
//   G p = w - grad q.
// In spectral form: column iFFT of (p1^, p2^, d^ = i kx p1^ + i ky p2^), one row kernel
// (C2R, pointwise w and q, R2C), column FFT whose epilogue forms (G p)^ = w^ - i k q^.
// A^{-1} per mode (Def:A): z = (r - alpha k (k.r) / (sigma + alpha |k|^2)) / sigma.
// The n/2 wavenumbers are 0 in both directions (§6.1).
#include <cstdio>
#include <vector>

#include "sgn_2d_dev.cuh"

namespace sgn {

using namespace d2;

namespace {

// ---- last-block reduction ------------------------------------------------------------
// Each block writes its partial sum; the last block to arrive sums them in a fixed order
// (deterministic) and runs `fin(total)` on thread 0.  float32 partials reduce across the
// block in double-float; only the block sums are float64.
template <int NT, typename Fin>
__device__ __forceinline__ void grid_finish(double s, double* parts, Scal2d* sc, Fin fin);

template <int NT, typename Fin>
__device__ __forceinline__ void grid_reduce(double v, double* parts, Scal2d* sc, Fin fin) {
  __shared__ double redb[NT / 32 + 1];
  grid_finish<NT>(block_sum<NT>(v, redb), parts, sc, fin);
}

template <int NT, typename Fin>
__device__ __forceinline__ void grid_reduce(float v, double* parts, Scal2d* sc, Fin fin) {
  __shared__ df slot[NT / 32];
  __shared__ double bs;
  block_sum_df<NT>(v, slot, [&](float hi, float lo) { bs = (double)hi + (double)lo; });
  grid_finish<NT>(bs, parts, sc, fin);
}

template <int NT, typename Fin>
__device__ __forceinline__ void grid_finish(double s, double* parts, Scal2d* sc, Fin fin) {
  __shared__ double red[NT / 32 + 1];
  __shared__ bool last;
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = s;
    __threadfence();
    unsigned int t = atomicAdd(&sc->ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += NT) acc += ((volatile double*)parts)[i];
    acc = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) {
      sc->ticket = 0;
      fin(acc);
      __threadfence();
    }
  }
}

// =======================================================================================
// Column pass: tiles of TW columns of K half planes, transposed into shared memory
// (column c of plane q at buf + (q TW + c) * (ny + 1)), transformed along y.
// =======================================================================================
enum ColMode { COL_FWD = 0, COL_INV = 1, COL_MATVEC_IN = 2, COL_MATVEC_OUT = 3 };

struct ColArgs {
  void* planes[4];          // K half planes (cplx<T>), in place unless noted
  int K;
  // COL_MATVEC_IN: input vector (2 half planes of cplx<TV>) and optional p update
  const void* vin[2];
  // COL_MATVEC_OUT: output G v (2 half planes) and the dot partner
  void* vout[2];
  const void* vdot[2];
  const void* bvec[2];      // residual mode: r = b - G x (high precision)
  int residual;             // 1: out = b - G v instead of G v
  Scal2d* sc;
  double* parts;
  int pupdate;              // COL_MATVEC_IN: p = A^{-1} r + beta p first (r in rin)
  void* pio[2];             // p planes (read/write) when pupdate
  const void* rin[2];
  int check_done;           // return immediately when sc->done
};

template <typename T, int TW, int MAXB, int MODE>
__global__ void __launch_bounds__(kColNT, 1) k2_cols(Modes2d M, int log2ny, const void* t64,
                                                     const void* t32, ColArgs a) {
  if (a.check_done && ((volatile Scal2d*)a.sc)->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem);
  const cplx<T>* tw = Tw<T>::get(t64, t32);
  const int ny = M.ny, H = M.H, stride = ny + 1;
  const int c0 = blockIdx.x * TW;
  const int nplanes = (MODE == COL_MATVEC_IN || MODE == COL_MATVEC_OUT) ? 3 : a.K;
  using TP = typename WorkP<T>::type;         // per-mode precision (float32 for float32)
  const ModesT<TP> MT(M);

  // ---- load
  for (int e = threadIdx.x; e < TW * ny; e += kColNT) {
    const int y = e / TW, c = e % TW, col = c0 + c;
    const long long gi = (long long)y * H + col;
    const bool ok = col < H;
    if constexpr (MODE == COL_MATVEC_IN) {
      cplx<T> p1 = mk(from_int<T>(0), from_int<T>(0)), p2 = p1;
      if (ok) {
        if (a.pupdate) {
          // p = A^{-1} r + beta p (the inner solve: T is float32 or float64)
          if constexpr (std::is_same<T, TP>::value) {
            cplx<T> r1 = ld_c<T>(a.rin[0], gi), r2 = ld_c<T>(a.rin[1], gi);
            cplx<T> q1 = ld_c<T>(a.pio[0], gi), q2 = ld_c<T>(a.pio[1], gi);
            const T beta = cg_beta(a.sc, T(0));
            cplx<T> z1, z2;
            ainv_of(a.sc, T(0)).apply(MT.kx(col), MT.ky(y), r1, r2, z1, z2);
            p1 = z1 + q1 * beta;
            p2 = z2 + q2 * beta;
          }
          st_c<T>(a.pio[0], gi, p1);
          st_c<T>(a.pio[1], gi, p2);
        } else {
          p1 = ld_c<T>(a.vin[0], gi);
          p2 = ld_c<T>(a.vin[1], gi);
        }
      }
      buf[(0 * TW + c) * stride + y] = p1;
      buf[(1 * TW + c) * stride + y] = p2;
    } else {
      for (int q = 0; q < nplanes; ++q)
        buf[(q * TW + c) * stride + y] = ok ? ld_c<T>(a.planes[q], gi)
                                            : mk(from_int<T>(0), from_int<T>(0));
    }
  }
  __syncthreads();
  if constexpr (MODE == COL_MATVEC_IN) {
    // A real field's half spectrum is Hermitian in ky on the kx = 0 and kx = nx/2 columns.
    // Rounding in the float32 inner solves leaves a small anti-Hermitian part there, which
    // the packed row C2R would leak between fields; project it out before the transform,
    // then form d^ = i kx p1^ + i ky p2^ from the projected vector.
    for (int c = 0; c < TW; ++c) {
      const int col = c0 + c;
      if (col != 0 && col != (M.nx >> 1)) continue;
      for (int q = 0; q < 2; ++q) {
        cplx<T>* v = buf + (q * TW + c) * stride;
        for (int y = threadIdx.x; y <= (ny >> 1); y += kColNT) {
          const int ym = (ny - y) & (ny - 1);
          cplx<T> a = v[y], b = conj(v[ym]);
          cplx<T> s = a + b;
          cplx<T> hm = mk(half(s.x), half(s.y));
          v[y] = hm;
          v[ym] = conj(hm);
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TW * ny; e += kColNT) {
      const int y = e / TW, c = e % TW, col = c0 + c;
      const T kx = mode_k<T>(MT, col < H ? col : (M.nx >> 1), true),
              ky = mode_k<T>(MT, y, false);
      buf[(2 * TW + c) * stride + y] =
          mul_ik(buf[(0 * TW + c) * stride + y], kx) + mul_ik(buf[(1 * TW + c) * stride + y], ky);
    }
    __syncthreads();
  }
  const bool inverse = (MODE == COL_INV || MODE == COL_MATVEC_IN);
  // the planes' columns lie at one stride (sequence q TW + c): one batched transform of all
  // of them, so every stage's butterflies spread over the whole CTA
  cta_fft_batch<T, kColNT, MAXB>(buf, ny, log2ny, nplanes * TW, stride, inverse, tw);

  // ---- store / epilogue
  if constexpr (MODE == COL_MATVEC_OUT) {
    const double sigma = a.sc ? a.sc->sigma : 0.0, alphaA = a.sc ? a.sc->alpha_A : 0.0;
    double part = 0.0;      // residual mode (double-float or float64 data)
    TP partw = 0;           // dot-product mode, in the working precision
    for (int e = threadIdx.x; e < TW * ny; e += kColNT) {
      const int y = e / TW, c = e % TW, col = c0 + c;
      if (col >= H) continue;
      const long long gi = (long long)y * H + col;
      const T kx = mode_k<T>(MT, col, true), ky = mode_k<T>(MT, y, false);
      cplx<T> w1 = buf[(0 * TW + c) * stride + y], w2 = buf[(1 * TW + c) * stride + y];
      cplx<T> qh = buf[(2 * TW + c) * stride + y];
      cplx<T> g1 = w1 - mul_ik(qh, kx), g2 = w2 - mul_ik(qh, ky);
      if (a.residual) {
        g1 = ld_c<T>(a.bvec[0], gi) - g1;
        g2 = ld_c<T>(a.bvec[1], gi) - g2;
        // r.A^{-1}r for the stopping test
        const double kxd = M.kx(col), kyd = M.ky(y);
        const double k2 = kxd * kxd + kyd * kyd;
        const double f = alphaA / (sigma + alphaA * k2);
        double r1x = to_f64(g1.x), r1y = to_f64(g1.y), r2x = to_f64(g2.x), r2y = to_f64(g2.y);
        double krx = kxd * r1x + kyd * r2x, kry = kxd * r1y + kyd * r2y;
        double z1x = (r1x - f * kxd * krx) / sigma, z1y = (r1y - f * kxd * kry) / sigma;
        double z2x = (r2x - f * kyd * krx) / sigma, z2y = (r2y - f * kyd * kry) / sigma;
        part += M.weight(col) * (r1x * z1x + r1y * z1y + r2x * z2x + r2y * z2y);
      } else if (a.vdot[0]) {
        if constexpr (std::is_same<T, TP>::value) {
          cplx<T> p1 = ld_c<T>(a.vdot[0], gi), p2 = ld_c<T>(a.vdot[1], gi);
          partw += MT.weight(col) * (p1.x * g1.x + p1.y * g1.y + p2.x * g2.x + p2.y * g2.y);
        }
      }
      st_c<T>(a.vout[0], gi, g1);
      st_c<T>(a.vout[1], gi, g2);
    }
    if (a.residual) {
      grid_reduce<kColNT>(part, a.parts, a.sc, [&](double s) { a.sc->rz64 = s; });
    } else if (a.vdot[0]) {
      grid_reduce<kColNT>(partw, a.parts, a.sc, [&](double s) {
        Scal2d* sc = a.sc;
        if (!(s > 0.0) || !isfinite(s)) {
          sc->status = SGN_ERR_BREAKDOWN;
          sc->done = 1;
        } else {
          sc->alpha = sc->rz / s;
          sc->alphaf = (float)sc->alpha;
        }
      });
    }
  } else {
    for (int e = threadIdx.x; e < TW * ny; e += kColNT) {
      const int y = e / TW, c = e % TW, col = c0 + c;
      if (col >= H) continue;
      const long long gi = (long long)y * H + col;
      for (int q = 0; q < nplanes; ++q) st_c<T>(a.planes[q], gi, buf[(q * TW + c) * stride + y]);
    }
  }
}

// =======================================================================================
// Row passes.  Two rows per block (y0 = 2b, y1 = 2b + 1).
// =======================================================================================

// coefficient planes: c11 = eta(1+hx^2), c12 = eta hx hy, c22 = eta(1+hy^2),
// c13 = eta^2 hx/2, c23 = eta^2 hy/2, c33 = eta^3/3 (Def:MatrixM); hi in float, the
// double-float remainder in lo.
template <typename T>
__device__ __forceinline__ void coef6(const float* hi, const float* lo, long long P, long long j,
                                      T c[6]);
template <>
__device__ __forceinline__ void coef6<float>(const float* hi, const float* lo, long long P,
                                             long long j, float c[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) c[q] = hi[q * P + j];
}
template <>
__device__ __forceinline__ void coef6<df>(const float* hi, const float* lo, long long P,
                                          long long j, df c[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) c[q] = df(hi[q * P + j], lo[q * P + j]);
}
template <>
__device__ __forceinline__ void coef6<double>(const float* hi, const float* lo, long long P,
                                              long long j, double c[6]) {
#pragma unroll
  for (int q = 0; q < 6; ++q) c[q] = (double)hi[q * P + j] + (double)lo[q * P + j];
}

// Matvec row kernel: planes t0, t1, t2 hold (after the column iFFT) the row half spectra of
// p1, p2, d.  C2R -> pointwise w1, w2, q -> R2C back into t0, t1, t2.  Optionally writes
// the real-space input (p1, p2) to xout (two planes of P doubles).
template <typename T, int MAXB>
__global__ void __launch_bounds__(kRowNT, 1) k2_rows_matvec(Modes2d M, int log2nx, long long P,
                                                            const void* t64, const void* t32,
                                                            void* t0, void* t1, void* t2,
                                                            const float* chi, const float* clo,
                                                            double* xout, Scal2d* sc,
                                                            int check_done) {
  if (check_done && ((volatile Scal2d*)sc)->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = M.nx, H = M.H;
  cplx<T>* z = reinterpret_cast<cplx<T>*>(smem);           // 3 rows of nx
  const cplx<T>* tw = Tw<T>::get(t64, t32);
  const int y0 = 2 * blockIdx.x, y1 = y0 + 1;
  cplx<T>* T0 = reinterpret_cast<cplx<T>*>(t0);
  cplx<T>* T1 = reinterpret_cast<cplx<T>*>(t1);
  cplx<T>* T2 = reinterpret_cast<cplx<T>*>(t2);
  load_c2r_pair<T>(z, T0 + (long long)y0 * H, T1 + (long long)y0 * H, nx, kRowNT);
  load_c2r_pair<T>(z + nx, T0 + (long long)y1 * H, T1 + (long long)y1 * H, nx, kRowNT);
  load_c2r_pair<T>(z + 2 * nx, T2 + (long long)y0 * H, T2 + (long long)y1 * H, nx, kRowNT);
  __syncthreads();
  cta_fft_batch<T, kRowNT, MAXB>(z, nx, log2nx, 3, nx, true, tw);
  const T inv = pow2_inv<T>(log2nx + (__ffs(M.ny) - 1));    // 1 / (nx ny), exact
  for (int x = threadIdx.x; x < nx; x += kRowNT) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int y = r ? y1 : y0;
      const long long j = (long long)y * nx + x;
      cplx<T> pp = z[r * nx + x];
      T p1 = pp.x * inv, p2 = pp.y * inv;
      T d = (r ? z[2 * nx + x].y : z[2 * nx + x].x) * inv;
      if (xout) {
        xout[j] = to_f64(p1);
        xout[P + j] = to_f64(p2);
      }
      T c[6];
      coef6<T>(chi, clo, P, j, c);
      T w1 = c[0] * p1 + c[1] * p2 + c[3] * d;
      T w2 = c[1] * p1 + c[2] * p2 + c[4] * d;
      T q = c[3] * p1 + c[4] * p2 + c[5] * d;
      z[r * nx + x] = mk(w1, w2);
      if (r) z[2 * nx + x].y = q; else z[2 * nx + x].x = q;
    }
  }
  __syncthreads();
  cta_fft_batch<T, kRowNT, MAXB>(z, nx, log2nx, 3, nx, false, tw);
  // split back into half rows: (w1, w2) of y0, (w1, w2) of y1, (q y0, q y1); the row FFT
  // results are read only here, so the splits may write the half planes directly.
  split_r2c_pair<T>(z, T0 + (long long)y0 * H, T1 + (long long)y0 * H, nx, kRowNT);
  split_r2c_pair<T>(z + nx, T0 + (long long)y1 * H, T1 + (long long)y1 * H, nx, kRowNT);
  split_r2c_pair<T>(z + 2 * nx, T2 + (long long)y0 * H, T2 + (long long)y1 * H, nx, kRowNT);
}

// R2C row pass of K/2 packed pairs of real planes (double storage): pair q packs
// (src[2q], src[2q+1]); half rows go to dst[2q], dst[2q+1].  `scale` multiplies the input.
template <typename T, int MAXB>
__global__ void __launch_bounds__(kRowNT, 1) k2_rows_r2c(Modes2d M, int log2nx, long long P,
                                                         const void* t64, const void* t32,
                                                         const double* s0, const double* s1,
                                                         const double* s2, const double* s3,
                                                         void* d0, void* d1, void* d2, void* d3,
                                                         int npairs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = M.nx, H = M.H;
  cplx<T>* z = reinterpret_cast<cplx<T>*>(smem);
  const cplx<T>* tw = Tw<T>::get(t64, t32);
  const int y = blockIdx.x;
  const double* src[4] = {s0, s1, s2, s3};
  void* dst[4] = {d0, d1, d2, d3};
  for (int q = 0; q < npairs; ++q)
    for (int x = threadIdx.x; x < nx; x += kRowNT) {
      const long long j = (long long)y * nx + x;
      const double a = src[2 * q] ? src[2 * q][j] : 0.0, b = src[2 * q + 1] ? src[2 * q + 1][j] : 0.0;
      z[q * nx + x] = mk(num<T>(a), num<T>(b));
    }
  __syncthreads();
  cta_fft_batch<T, kRowNT, MAXB>(z, nx, log2nx, npairs, nx, false, tw);
  for (int q = 0; q < npairs; ++q)
    split_r2c_pair<T>(z + q * nx, reinterpret_cast<cplx<T>*>(dst[2 * q]) + (long long)y * H,
                      reinterpret_cast<cplx<T>*>(dst[2 * q + 1]) + (long long)y * H, nx, kRowNT);
}

// C2R row pass: pair q of half planes (src[2q], src[2q+1]) -> real planes dst[2q],
// dst[2q+1] (double storage), scaled by 1/(nx ny).
template <typename T, int MAXB>
__global__ void __launch_bounds__(kRowNT, 1) k2_rows_c2r(Modes2d M, int log2nx, long long P,
                                                         const void* t64, const void* t32,
                                                         const void* s0, const void* s1,
                                                         const void* s2, const void* s3,
                                                         double* d0, double* d1, double* d2,
                                                         double* d3, int npairs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = M.nx, H = M.H;
  cplx<T>* z = reinterpret_cast<cplx<T>*>(smem);
  const cplx<T>* tw = Tw<T>::get(t64, t32);
  const int y = blockIdx.x;
  const void* src[4] = {s0, s1, s2, s3};
  double* dst[4] = {d0, d1, d2, d3};
  for (int q = 0; q < npairs; ++q)
    load_c2r_pair<T>(z + q * nx, reinterpret_cast<const cplx<T>*>(src[2 * q]) + (long long)y * H,
                     reinterpret_cast<const cplx<T>*>(src[2 * q + 1]) + (long long)y * H, nx,
                     kRowNT);
  __syncthreads();
  cta_fft_batch<T, kRowNT, MAXB>(z, nx, log2nx, npairs, nx, true, tw);
  const T inv = pow2_inv<T>(log2nx + (__ffs(M.ny) - 1));    // 1 / (nx ny), exact
  for (int q = 0; q < npairs; ++q)
    for (int x = threadIdx.x; x < nx; x += kRowNT) {
      const long long j = (long long)y * nx + x;
      cplx<T> v = z[q * nx + x];
      if (dst[2 * q]) dst[2 * q][j] = to_f64(v.x * inv);
      if (dst[2 * q + 1]) dst[2 * q + 1][j] = to_f64(v.y * inv);
    }
}

// =======================================================================================
// Per-mode kernels over half spectra
// =======================================================================================

// Spectral ops for derivatives and A^{-1}:
//   OP_GRAD: out0 = i kx in0, out1 = i ky in0 (and out2, out3 from in1)
//   OP_AINV: (out0, out1) = A^{-1} (in0, in1)
//   OP_DIV : out0 = i kx in0 + i ky in1
enum SpecOp { OP_GRAD = 0, OP_AINV = 1 };

template <typename T, int OP>
__global__ void k2_spec(Modes2d M, const void* in0, const void* in1, void* out0, void* out1,
                        void* out2, void* out3, const Scal2d* sc, const SolveRec* A) {
  const long long HP = (long long)M.ny * M.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    const double kx = M.kx(c), ky = M.ky(y);
    if constexpr (OP == OP_GRAD) {
      cplx<T> a = ld_c<T>(in0, i);
      st_c<T>(out0, i, mul_ik(a, num<T>(kx)));
      st_c<T>(out1, i, mul_ik(a, num<T>(ky)));
      if (in1) {
        cplx<T> b = ld_c<T>(in1, i);
        st_c<T>(out2, i, mul_ik(b, num<T>(kx)));
        st_c<T>(out3, i, mul_ik(b, num<T>(ky)));
      }
    } else {
      const double sigma = A ? A->sigma : sc->sigma, alpha = A ? A->alpha : sc->alpha_A;
      const double f = alpha / (sigma + alpha * (kx * kx + ky * ky));
      const T kxT = num<T>(kx), kyT = num<T>(ky), fT = num<T>(f), is = num<T>(1.0 / sigma);
      cplx<T> r1 = ld_c<T>(in0, i), r2 = ld_c<T>(in1, i);
      cplx<T> kr = r1 * kxT + r2 * kyT;
      st_c<T>(out0, i, (r1 - kr * (fT * kxT)) * is);
      st_c<T>(out1, i, (r2 - kr * (fT * kyT)) * is);
    }
  }
}

// Spectral combinations of the 2d right-hand side (i k multiplies by the wavenumber, the
// Nyquist wavenumbers being 0):
//   RHS_DIVD: out0 = d^ = i kx in0 + i ky in1 (d = div u), out1 = i kx in2 + i ky in3
//             (m = div(eta u)), out2 = i kx d^, out3 = i ky d^ (grad d);
//   RHS_DIV2: out0 = i kx in0 + i ky in1, out1 = i kx in1 + i ky in2 (the two components of
//             div(eta u (x) u) from eta u u, eta u v, eta v v).
enum RhsSpec { RHS_DIVD = 0, RHS_DIV2 = 1 };
template <typename T, int MODE>
__global__ void k2_spec_rhs(Modes2d M, const void* in0, const void* in1, const void* in2,
                            const void* in3, void* out0, void* out1, void* out2, void* out3) {
  const long long HP = (long long)M.ny * M.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    const T kx = num<T>(M.kx(c)), ky = num<T>(M.ky(y));
    const cplx<T> a = ld_c<T>(in0, i), b = ld_c<T>(in1, i), e = ld_c<T>(in2, i);
    if constexpr (MODE == RHS_DIVD) {
      const cplx<T> dh = mul_ik(a, kx) + mul_ik(b, ky);
      st_c<T>(out0, i, dh);
      st_c<T>(out1, i, mul_ik(e, kx) + mul_ik(ld_c<T>(in3, i), ky));
      st_c<T>(out2, i, mul_ik(dh, kx));
      st_c<T>(out3, i, mul_ik(dh, ky));
    } else {
      st_c<T>(out0, i, mul_ik(a, kx) + mul_ik(b, ky));
      st_c<T>(out1, i, mul_ik(b, kx) + mul_ik(e, ky));
    }
  }
}

// Inner PCG update: x += alpha p; r -= alpha g; rz = r.A^{-1}r; last block forms beta and
// the stopping decision.
// In a solve graph (use_h) it also sets the inner loop's condition: 0 once done, which
// covers a breakdown found by the matvec (done already set: every block returns at once,
// and block 0 ends the loop), so the loop cannot outlive the iteration cap.
template <typename T>
__global__ void __launch_bounds__(256) k2_update(Modes2d M, void* x1, void* x2, void* r1p,
                                                 void* r2p, const void* p1p, const void* p2p,
                                                 const void* g1p, const void* g2p, Scal2d* sc,
                                                 double* parts, cudaGraphConditionalHandle hin,
                                                 int use_h) {
  if (((volatile Scal2d*)sc)->done) {
    if (use_h && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hin, 0u);
    return;
  }
  const long long HP = (long long)M.ny * M.H;
  const ModesT<T> MT(M);
  const AinvT<T> Ai = ainv_of(sc, T(0));
  const T a = cg_alpha(sc, T(0));
  T part = 0;
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < HP; i += (long long)gridDim.x * 256) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    cplx<T> p1 = ld_c<T>(p1p, i), p2 = ld_c<T>(p2p, i);
    st_c<T>(x1, i, ld_c<T>(x1, i) + p1 * a);
    st_c<T>(x2, i, ld_c<T>(x2, i) + p2 * a);
    cplx<T> r1 = ld_c<T>(r1p, i) - ld_c<T>(g1p, i) * a;
    cplx<T> r2 = ld_c<T>(r2p, i) - ld_c<T>(g2p, i) * a;
    st_c<T>(r1p, i, r1);
    st_c<T>(r2p, i, r2);
    cplx<T> z1, z2;
    Ai.apply(MT.kx(c), MT.ky(y), r1, r2, z1, z2);
    part += MT.weight(c) * (r1.x * z1.x + r1.y * z1.y + r2.x * z2.x + r2.y * z2.y);
  }
  grid_reduce<256>(part, parts, sc, [&](double rz_new) {
    sc->iters += 1;
    if (!isfinite(rz_new)) {
      sc->status = SGN_ERR_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->beta = rz_new / sc->rz;
      sc->betaf = (float)sc->beta;
      sc->rz = rz_new;
      if (sqrt(rz_new) <= sc->tol) {
        sc->done = 1;
      } else if (sc->iters >= sc->cap) {
        sc->status = SGN_ERR_NOT_CONVERGED;
        sc->done = 1;
      }
    }
    if (use_h) cudaGraphSetConditional(hin, sc->done ? 0u : 1u);
  });
}

// Start of an inner solve: r = scale * src (high -> T), x = 0, p = 0, beta = 0,
// rz = r.A^{-1}r (last block), done if already below tol.
// scale_sc: scale = 1 / sc->rn (the solve graph); use_h: set the inner loop's condition.
// A solve whose status is already an error starts done.
template <typename TH, typename T>
__global__ void __launch_bounds__(256) k2_inner_start(Modes2d M, const void* s1, const void* s2,
                                                      double scale, void* r1p, void* r2p,
                                                      void* x1, void* x2, void* p1, void* p2,
                                                      Scal2d* sc, double* parts, int scale_sc,
                                                      cudaGraphConditionalHandle hin, int use_h,
                                                      int cm) {
  const long long HP = (long long)M.ny * M.H;
  const ModesT<T> MT(M);
  const AinvT<T> Ai = ainv_of(sc, T(0));
  const T sc_t = (T)(scale_sc ? 1.0 / sc->rn : scale);
  T part = 0;
  const cplx<T> zero = mk(T(0), T(0));
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < HP; i += (long long)gridDim.x * 256) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    cplx<TH> a = ld_c<TH>(s1, i), b = ld_c<TH>(s2, i);
    cplx<T> r1 = mk(to_work<T>(a.x) * sc_t, to_work<T>(a.y) * sc_t);
    cplx<T> r2 = mk(to_work<T>(b.x) * sc_t, to_work<T>(b.y) * sc_t);
    // cm: the persistent inner solve keeps r, p, d column-major ([H][ny])
    const long long o = cm ? (long long)c * M.ny + y : i;
    st_c<T>(r1p, o, r1);
    st_c<T>(r2p, o, r2);
    st_c<T>(x1, i, zero);
    st_c<T>(x2, i, zero);
    st_c<T>(p1, i, zero);
    st_c<T>(p2, i, zero);
    cplx<T> z1, z2;
    Ai.apply(MT.kx(c), MT.ky(y), r1, r2, z1, z2);
    part += MT.weight(c) * (r1.x * z1.x + r1.y * z1.y + r2.x * z2.x + r2.y * z2.y);
  }
  grid_reduce<256>(part, parts, sc, [&](double rz) {
    sc->rz = rz;
    sc->beta = 0.0;
    sc->betaf = 0.0f;
    sc->done = (sc->status != SGN_OK || sqrt(rz) <= sc->tol) ? 1 : 0;
    if (use_h) cudaGraphSetConditional(hin, sc->done ? 0u : 1u);
  });
}

// x_high += scale * d (T -> high precision); cm: d is column-major ([H][ny])
template <typename TH, typename T>
__global__ void k2_accumulate(Modes2d M, void* x1, void* x2, const void* d1, const void* d2,
                              double scale, const Scal2d* sc, int cm) {   // sc: scale = sc->rn
  const long long HP = (long long)M.ny * M.H;
  const TH s = num<TH>(sc ? sc->rn : scale);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;
    const long long o = cm ? (long long)c * M.ny + y : i;
    cplx<T> a = ld_c<T>(d1, o), b = ld_c<T>(d2, o);
    cplx<TH> u = ld_c<TH>(x1, i), v = ld_c<TH>(x2, i);
    st_c<TH>(x1, i, mk(u.x + widen<TH>(a.x) * s, u.y + widen<TH>(a.y) * s));
    st_c<TH>(x2, i, mk(v.x + widen<TH>(b.x) * s, v.y + widen<TH>(b.y) * s));
  }
}

// b.A^{-1}b for a vector of two half planes (high precision) -> sc->bb
template <typename TH>
__global__ void __launch_bounds__(256) k2_bnorm(Modes2d M, const void* b1, const void* b2,
                                                Scal2d* sc, double* parts) {
  const long long HP = (long long)M.ny * M.H;
  const double sigma = sc->sigma, alphaA = sc->alpha_A;
  double part = 0.0;
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < HP; i += (long long)gridDim.x * 256) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    const double kx = M.kx(c), ky = M.ky(y);
    cplx<TH> a = ld_c<TH>(b1, i), b = ld_c<TH>(b2, i);
    const double f = alphaA / (sigma + alphaA * (kx * kx + ky * ky));
    double r1x = to_f64(a.x), r1y = to_f64(a.y), r2x = to_f64(b.x), r2y = to_f64(b.y);
    double krx = kx * r1x + ky * r2x, kry = kx * r1y + ky * r2y;
    part += M.weight(c) * ((r1x * (r1x - f * kx * krx) + r1y * (r1y - f * kx * kry) +
                            r2x * (r2x - f * ky * krx) + r2y * (r2y - f * ky * kry)) / sigma);
  }
  grid_reduce<256>(part, parts, sc, [&](double s) { sc->bb = s; });
}

// coefficient planes (Def:MatrixM) from eta, grad h
// (and float32 eta, h_x, h_y for the persistent inner solve, which forms its coefficients
// from them)
__global__ void k2_coef_planes(long long P, const double* eta, const double* gh, float* hi,
                               float* lo, float* ehh) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < P;
       j += (long long)gridDim.x * blockDim.x) {
    const double e = eta[j], hx = gh[j], hy = gh[P + j];
    ehh[j] = (float)e;
    ehh[P + j] = (float)hx;
    ehh[2 * P + j] = (float)hy;
    const double c[6] = {e * (1.0 + hx * hx), e * hx * hy, e * (1.0 + hy * hy), 0.5 * e * e * hx,
                         0.5 * e * e * hy, e * e * e / 3.0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float h = (float)c[q];
      hi[q * P + j] = h;
      lo[q * P + j] = (float)(c[q] - (double)h);
    }
  }
}

// a1 in 2d: block reductions of eta_min, eta_max, max |grad h|^2, max eta(1 + l+ |grad h|^2)
__global__ void __launch_bounds__(256) k2_coeffs(long long P, const double* eta, const double* gh,
                                                 int kind, double* parts, Scal2d* sc,
                                                 SolveRec* rec) {
  __shared__ double red[256 / 32 + 1];
  double emin = 1e308, emax = -1e308, g2max = 0.0, sopt = -1e308, bad = 0.0;
  for (long long j = blockIdx.x * 256ll + threadIdx.x; j < P; j += (long long)gridDim.x * 256) {
    const double e = eta[j], hx = gh[j], hy = gh[P + j], g2 = hx * hx + hy * hy;
    if (!(e > 0.0) || !(g2 < 1e300)) bad = 1.0;
    emin = fmin(emin, e);
    emax = fmax(emax, e);
    g2max = fmax(g2max, g2);
    sopt = fmax(sopt, e + kLambdaPlus * e * g2);
  }
  emin = block_min<256>(emin, red);
  emax = block_max<256>(emax, red);
  g2max = block_max<256>(g2max, red);
  sopt = block_max<256>(sopt, red);
  bad = block_max<256>(bad, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double* p = parts + 5 * blockIdx.x;
    p[0] = emin;
    p[1] = emax;
    p[2] = g2max;
    p[3] = sopt;
    p[4] = bad;
    __threadfence();
    last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  {
    // the last block reduces the per-block partials with all its threads
    volatile double* vp = parts;
    double a = 1e308, b = -1e308, g = 0.0, s = -1e308, bd = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) {
      a = fmin(a, vp[5 * i]);
      b = fmax(b, vp[5 * i + 1]);
      g = fmax(g, vp[5 * i + 2]);
      s = fmax(s, vp[5 * i + 3]);
      bd = fmax(bd, vp[5 * i + 4]);
    }
    a = block_min<256>(a, red);
    b = block_max<256>(b, red);
    g = block_max<256>(g, red);
    s = block_max<256>(s, red);
    bd = block_max<256>(bd, red);
    if (threadIdx.x != 0) return;
    sc->ticket = 0;
    if (kind < 0) kind = sc->kind;          // the solve graph passes the kind through sc
    SolveRec R = {};
    R.eta_min = a;
    R.eta_max = b;
    if (bd > 0.0) {
      R.status = SGN_ERR_NONPOSITIVE_DEPTH;
    } else {
      const double ratio3 = (b / a) * (b / a) * (b / a);
      R.flat = sqrt(g) <= kFlatSlope;
      if (R.flat) {
        R.sigma = b;
        R.alpha = b * b * b / 3.0;
        R.kappa_ub = ratio3;
      } else if (kind == SGN_COEF_OPT) {
        R.sigma = s;
        R.alpha = kLambdaPlus * b * b * b;
        R.kappa_ub = fmax(s / a, (kLambdaPlus / kLambdaMinus) * ratio3);
      } else {
        R.sigma = b * (1.0 + kLambdaPlus * g);
        R.alpha = kLambdaPlus * b * b * b;
        R.kappa_ub = fmax((b / a) * (1.0 + kLambdaPlus * g), (kLambdaPlus / kLambdaMinus) * ratio3);
      }
      R.status = SGN_OK;
    }
    if (rec) *rec = R;
    sc->sigma = R.sigma;
    sc->alpha_A = R.alpha;
    sc->sigf = (float)R.sigma;
    sc->alphaAf = (float)R.alpha;
    sc->isigf = (float)(1.0 / R.sigma);
    sc->kappa_ub = R.kappa_ub;
    sc->eta_min = R.eta_min;
    sc->eta_max = R.eta_max;
    sc->flat = R.flat;
    sc->status = R.status;
    __threadfence();
  }
}

__global__ void k2_set_given(Scal2d* sc, const SolveRec* g) {
  sc->sigma = g->sigma;
  sc->alpha_A = g->alpha;
  sc->sigf = (float)g->sigma;
  sc->alphaAf = (float)g->alpha;
  sc->isigf = (float)(1.0 / g->sigma);
  sc->kappa_ub = g->kappa_ub;
  sc->flat = g->flat;
  sc->status = SGN_OK;
}

__global__ void k2_report(const Scal2d* sc, SolveRec* rec, int refinements) {   // < 0: sc's
  if (refinements < 0) refinements = sc->refinements;
  SolveRec R = {};
  R.sigma = sc->sigma;
  R.alpha = sc->alpha_A;
  R.kappa_ub = sc->kappa_ub;
  R.eta_min = sc->eta_min;
  R.eta_max = sc->eta_max;
  R.flat = sc->flat;
  R.iters = sc->iters;
  R.refinements = refinements;
  R.ratio = sc->bb > 0.0 ? sqrt(fmax(sc->rz64, 0.0) / sc->bb) : 0.0;
  R.status = sc->status;
  *rec = R;
}

__global__ void k2_lincomb(long long n, double* out, const double* x0, const double* x1,
                           const double* x2, const double* x3, double a0, double a1, double a2,
                           double a3, int nx, const double* f0, const double* f1, const double* f2,
                           const double* f3, double c0, double c1, double c2, double c3, int nf,
                           const double* dt) {
  const double d = dt[0];
  const double* X[4] = {x0, x1, x2, x3};
  const double A[4] = {a0, a1, a2, a3};
  const double* F[4] = {f0, f1, f2, f3};
  const double Cc[4] = {c0, c1, c2, c3};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0, accf = 0.0;
    for (int t = 0; t < nx; ++t) acc += A[t] * X[t][i];
    for (int t = 0; t < nf; ++t) accf += Cc[t] * F[t][i];
    out[i] = acc + d * accf;
  }
}

// RHS pointwise stages (T arithmetic, double storage), see launch_rhs2d.
template <typename T>
__global__ void k2_rhs_stage(int stage, long long P, double g, const double* eta, const double* u,
                             const double* hgt, const double* gh, double* w, double* f_eta,
                             double* f_U) {
  // w: scratch planes [0..]; see launch_rhs2d for the meaning of each index
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < P;
       j += (long long)gridDim.x * blockDim.x) {
    const T e = num<T>(eta[j]), uu = num<T>(u[j]), vv = num<T>(u[P + j]);
    const T hx = num<T>(gh[j]), hy = num<T>(gh[P + j]);
    if (stage == 0) {
      // inputs for the first derivative passes
      w[0 * P + j] = to_f64(e * uu);                       // eta u
      w[1 * P + j] = to_f64(e * vv);                       // eta v
      w[2 * P + j] = eta[j] - hgt[j];                      // zeta
      w[3 * P + j] = to_f64(hx * uu + hy * vv);            // s
      w[4 * P + j] = to_f64(e * uu * uu);                  // eta u u
      w[5 * P + j] = to_f64(e * uu * vv);                  // eta u v
      w[6 * P + j] = to_f64(e * vv * vv);                  // eta v v
    } else {
      // 7 d = div u, 14 m = div(eta u), 18 zeta_x, 19 zeta_y, 20 s_x, 21 s_y, 22 d_x, 23 d_y,
      // 24 and 26 the x and y components of div(eta u (x) u); Phi -> 8, Psi -> 9
      const T d = num<T>(w[7 * P + j]);
      const T m = num<T>(w[14 * P + j]);
      const T s = hx * uu + hy * vv;
      const T Sv = uu * num<T>(w[20 * P + j]) + vv * num<T>(w[21 * P + j]);
      const T Q = uu * num<T>(w[22 * P + j]) + vv * num<T>(w[23 * P + j]) - d * d;
      const T e2 = e * e, md = m * d;
      if (stage == 2) {
        w[8 * P + j] = to_f64(e2 * e * Q * num<T>(1.0 / 3.0) + e2 * md + half(e2 * Sv) + e * m * s);
        w[9 * P + j] = to_f64(half(e2 * Q) + e * md + e * Sv + m * s);
      } else {
        // stage 3: Phi_x -> 30, Phi_y -> 31
        const T Psi = num<T>(w[9 * P + j]);
        const T gT = num<T>(g);
        f_eta[j] = -to_f64(m);
        const T fx = num<T>(w[30 * P + j]) - gT * e * num<T>(w[18 * P + j]) -
                     num<T>(w[24 * P + j]) - hx * Psi;
        const T fy = num<T>(w[31 * P + j]) - gT * e * num<T>(w[19 * P + j]) -
                     num<T>(w[26 * P + j]) - hy * Psi;
        f_U[j] = to_f64(fx);
        f_U[P + j] = to_f64(fy);
      }
    }
  }
}

// SBDF2 residual in spectral form: res = A u - G u + U with A u = sigma u + alpha k (k.u)
template <typename T>
__global__ void k2_linimp_combine(Modes2d M, const SolveRec* A, const void* u1, const void* u2,
                                  const void* g1, const void* g2, const void* U1, const void* U2,
                                  void* o1, void* o2) {
  const long long HP = (long long)M.ny * M.H;
  const double sigma = A->sigma, alpha = A->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;   // half planes < 2^31 elements
    const T kx = num<T>(M.kx(c)), ky = num<T>(M.ky(y));
    cplx<T> a = ld_c<T>(u1, i), b = ld_c<T>(u2, i);
    cplx<T> ku = a * kx + b * ky;
    const T s = num<T>(sigma), al = num<T>(alpha);
    st_c<T>(o1, i, a * s + ku * (al * kx) - ld_c<T>(g1, i) + ld_c<T>(U1, i));
    st_c<T>(o2, i, b * s + ku * (al * ky) - ld_c<T>(g2, i) + ld_c<T>(U2, i));
  }
}

template <typename T>
__global__ void k2_axpby(long long HP, void* o1, void* o2, const void* a1, const void* a2,
                         const void* b1, const void* b2, double ca, double cb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const T A = num<T>(ca), B = num<T>(cb);
    st_c<T>(o1, i, ld_c<T>(a1, i) * A + ld_c<T>(b1, i) * B);
    st_c<T>(o2, i, ld_c<T>(a2, i) * A + ld_c<T>(b2, i) * B);
  }
}

// ---------------------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------------------

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
  return raise_smem(kernel, bytes);
}

// Columns per CTA for this layout: 2, or 4 for float32 planes when 2-column tiles would not
// fit one wave on 152 SMs (nx = 1024: 257 tiles).  Four float32 columns also fill each
// 32-byte sector of a row (two leave half of it unread); wider elements fill it with two.
template <typename T>
int col_tw_of(const Layout2d& L) {
  const int H = L.nx / 2 + 1;
  return (std::is_same<T, float>::value && (H + 1) / 2 > 152) ? 4 : 2;
}

template <typename T>
size_t col_smem(const Layout2d& L, int K) {
  return (size_t)K * col_tw_of<T>(L) * (L.ny + 1) * sizeof(cplx<T>);
}

template <typename T>
size_t row_smem(const Layout2d& L, int nrows) {
  return (size_t)nrows * L.nx * sizeof(cplx<T>);
}

// column pass launcher: MAXB from the K planes' TW columns x ny/4 butterflies per radix-4
// stage over kColNT threads
template <typename T, int TW, int MODE>
cudaError_t cols_tw(const Layout2d& L, const void* t64, const void* t32, const ColArgs& a,
                    cudaStream_t s) {
  const Modes2d M = modes_of(L);
  const int tiles = (M.H + TW - 1) / TW;
  const int K = (MODE == COL_MATVEC_IN || MODE == COL_MATVEC_OUT) ? 3 : a.K;
  const size_t sm = (size_t)K * TW * (L.ny + 1) * sizeof(cplx<T>);
  // K TW ny / 4 butterflies per radix-4 stage; MAXB = ceil(that / kColNT): at most 4, or 8
  // for the four float32 columns of the widest grids
  const int need = (K * TW * L.ny / 4 + kColNT - 1) / kColNT;
  cudaError_t e;
  if (need <= 1) {
    auto k = k2_cols<T, TW, 1, MODE>;
    if ((e = smem_attr(k, sm))) return e;
    k<<<tiles, kColNT, sm, s>>>(M, L.ly, t64, t32, a);
  } else if (need <= 2) {
    auto k = k2_cols<T, TW, 2, MODE>;
    if ((e = smem_attr(k, sm))) return e;
    k<<<tiles, kColNT, sm, s>>>(M, L.ly, t64, t32, a);
  } else if (need <= 4 || TW < 4) {
    auto k = k2_cols<T, TW, 4, MODE>;
    if ((e = smem_attr(k, sm))) return e;
    k<<<tiles, kColNT, sm, s>>>(M, L.ly, t64, t32, a);
  } else {
    if constexpr (TW == 4) {
      auto k = k2_cols<T, TW, 8, MODE>;
      if ((e = smem_attr(k, sm))) return e;
      k<<<tiles, kColNT, sm, s>>>(M, L.ly, t64, t32, a);
    }
  }
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t cols(const Layout2d& L, const void* t64, const void* t32, const ColArgs& a,
                 cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (col_tw_of<T>(L) == 4) return cols_tw<T, 4, MODE>(L, t64, t32, a, s);
  }
  return cols_tw<T, 2, MODE>(L, t64, t32, a, s);
}

template <typename T>
cudaError_t rows_matvec(const Layout2d& L, const void* t64, const void* t32, void* t0, void* t1,
                        void* t2, double* xout, Scal2d* sc, int check_done, cudaStream_t s) {
  const Modes2d M = modes_of(L);
  const size_t sm = row_smem<T>(L, 3);
  const int need = (3 * L.nx / 4 + kRowNT - 1) / kRowNT;   // butterflies per thread
  cudaError_t e;
#define SGN_ROWS_MV(MB)                                                                     \
  {                                                                                        \
    auto k = k2_rows_matvec<T, MB>;                                                        \
    if ((e = smem_attr(k, sm))) return e;                                                  \
    k<<<L.ny / 2, kRowNT, sm, s>>>(M, L.lx, L.P, t64, t32, t0, t1, t2, L.coef,              \
                                   L.coef_lo, xout, sc, check_done);                       \
  }
  if (need <= 1) SGN_ROWS_MV(1) else if (need <= 2) SGN_ROWS_MV(2) else if (need <= 3) SGN_ROWS_MV(3)
  else SGN_ROWS_MV(4)
#undef SGN_ROWS_MV
  return cudaGetLastError();
}

template <typename T>
cudaError_t rows_r2c(const Layout2d& L, const void* t64, const void* t32, const double* s0,
                     const double* s1, const double* s2, const double* s3, void* d0, void* d1,
                     void* d2, void* d3, int npairs, cudaStream_t s) {
  const Modes2d M = modes_of(L);
  const size_t sm = row_smem<T>(L, npairs);
  const int need = (npairs * L.nx / 4 + kRowNT - 1) / kRowNT;
  cudaError_t e;
#define SGN_ROWS_F(MB)                                                                       \
  {                                                                                         \
    auto k = k2_rows_r2c<T, MB>;                                                            \
    if ((e = smem_attr(k, sm))) return e;                                                   \
    k<<<L.ny, kRowNT, sm, s>>>(M, L.lx, L.P, t64, t32, s0, s1, s2, s3, d0, d1, d2, d3, npairs); \
  }
  if (need <= 1) SGN_ROWS_F(1) else if (need <= 2) SGN_ROWS_F(2) else SGN_ROWS_F(4)
#undef SGN_ROWS_F
  return cudaGetLastError();
}

template <typename T>
cudaError_t rows_c2r(const Layout2d& L, const void* t64, const void* t32, const void* s0,
                     const void* s1, const void* s2, const void* s3, double* d0, double* d1,
                     double* d2, double* d3, int npairs, cudaStream_t s) {
  const Modes2d M = modes_of(L);
  const size_t sm = row_smem<T>(L, npairs);
  const int need = (npairs * L.nx / 4 + kRowNT - 1) / kRowNT;
  cudaError_t e;
#define SGN_ROWS_I(MB)                                                                       \
  {                                                                                         \
    auto k = k2_rows_c2r<T, MB>;                                                            \
    if ((e = smem_attr(k, sm))) return e;                                                   \
    k<<<L.ny, kRowNT, sm, s>>>(M, L.lx, L.P, t64, t32, s0, s1, s2, s3, d0, d1, d2, d3, npairs); \
  }
  if (need <= 1) SGN_ROWS_I(1) else if (need <= 2) SGN_ROWS_I(2) else SGN_ROWS_I(4)
#undef SGN_ROWS_I
  return cudaGetLastError();
}

// half-plane slot q of the workspace (16 bytes per element)
inline void* slot(const Layout2d& L, int q) {
  return static_cast<char*>(L.vec) + (size_t)q * L.HP * 16;
}
inline void* tplane(const Layout2d& L, int q) {
  return static_cast<char*>(L.tp) + (size_t)q * L.HP * 16;
}

int grid_for(long long n, int nt) {
  long long b = (n + nt - 1) / nt;
  if (b > kMaxParts) b = kMaxParts;
  return (int)(b < 1 ? 1 : b);
}

// Forward transform of a real vector field (2 planes of P doubles) into 2 half planes.
template <typename T>
cudaError_t r2c_vec(const Layout2d& L, const void* t64, const void* t32, const double* v,
                    void* o1, void* o2, cudaStream_t s) {
  cudaError_t e = rows_r2c<T>(L, t64, t32, v, v + L.P, nullptr, nullptr, o1, o2, nullptr, nullptr,
                              1, s);
  if (e) return e;
  ColArgs a{};
  a.planes[0] = o1;
  a.planes[1] = o2;
  a.K = 2;
  return cols<T, COL_FWD>(L, t64, t32, a, s);
}

// Inverse transform of 2 half planes into a real vector field (the half planes are
// transformed in place along y first).
template <typename T>
cudaError_t c2r_vec(const Layout2d& L, const void* t64, const void* t32, void* i1, void* i2,
                    double* v, cudaStream_t s) {
  ColArgs a{};
  a.planes[0] = i1;
  a.planes[1] = i2;
  a.K = 2;
  cudaError_t e = cols<T, COL_INV>(L, t64, t32, a, s);
  if (e) return e;
  return rows_c2r<T>(L, t64, t32, i1, i2, nullptr, nullptr, v, v + L.P, nullptr, nullptr, 1, s);
}

// One spectral matvec: (g1, g2) = G (v1, v2) (or b - G v when residual) in precision T.
// Uses the 3 transform planes.  xout (nullable): real-space v on the way.
template <typename T>
cudaError_t matvec(const Layout2d& L, const void* t64, const void* t32, const void* v1,
                   const void* v2, void* g1, void* g2, const void* dot1, const void* dot2,
                   const void* b1, const void* b2, int residual, double* xout, Scal2d* sc,
                   int check_done, int pupdate, void* p1, void* p2, const void* r1,
                   const void* r2, cudaStream_t s) {
  ColArgs a{};
  a.planes[0] = tplane(L, 0);
  a.planes[1] = tplane(L, 1);
  a.planes[2] = tplane(L, 2);
  a.K = 3;
  a.vin[0] = v1;
  a.vin[1] = v2;
  a.sc = sc;
  a.parts = L.parts;
  a.check_done = check_done;
  a.pupdate = pupdate;
  a.pio[0] = p1;
  a.pio[1] = p2;
  a.rin[0] = r1;
  a.rin[1] = r2;
  // the column kernel writes its results into the transform planes
  ColArgs ain = a;
  cudaError_t e = cols<T, COL_MATVEC_IN>(L, t64, t32, ain, s);
  if (e) return e;
  if ((e = rows_matvec<T>(L, t64, t32, tplane(L, 0), tplane(L, 1), tplane(L, 2), xout, sc,
                          check_done, s)))
    return e;
  ColArgs aout = a;
  aout.vout[0] = g1;
  aout.vout[1] = g2;
  aout.vdot[0] = dot1;
  aout.vdot[1] = dot2;
  aout.bvec[0] = b1;
  aout.bvec[1] = b2;
  aout.residual = residual;
  return cols<T, COL_MATVEC_OUT>(L, t64, t32, aout, s);
}

}  // namespace

// =======================================================================================
// Layout
// =======================================================================================

namespace {

// The persistent inner solve's view of one instance: correction d^ (slots 8-9), r^ (4-5),
// p^ (6-7) and the first three transform planes, as float32 half planes.
PInst2d pinst_of(const Layout2d& L) {
  PInst2d pi;
  auto fp = [&](int q) { return reinterpret_cast<cplx<float>*>(slot(L, q)); };
  pi.x[0] = fp(8);
  pi.x[1] = fp(9);
  pi.r[0] = fp(4);
  pi.r[1] = fp(5);
  pi.p[0] = fp(6);
  pi.p[1] = fp(7);
  for (int q = 0; q < 3; ++q) pi.t[q] = reinterpret_cast<cplx<float>*>(tplane(L, q));
  pi.ehh = L.ehh;
  pi.sc = L.sc;
  pi.kxu = 2.0 * kPi / L.Lx;
  pi.kyu = 2.0 * kPi / L.Ly;
  return pi;
}

}  // namespace

// The cached solve graphs and their source graphs (kept until the executable graph goes).
void drop_solve_graphs(const Layout2d& L) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      if (L.solve_exec[i][j]) cudaGraphExecDestroy(L.solve_exec[i][j]);
      if (L.solve_graph[i][j]) cudaGraphDestroy(L.solve_graph[i][j]);
      L.solve_exec[i][j] = nullptr;
      L.solve_graph[i][j] = nullptr;
    }
}

// Appends a while node after the work captured so far on `cs` (which keeps capturing after
// it) and returns the node's body graph.
cudaError_t capture_add_while(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, &edges, &nd);
  if (e) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, edges, nd, &p))) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies);
}

cudaError_t layout2d_create(Layout2d& L, const sgn_grid& g) {
  L.nx = g.nx;
  L.ny = g.ny;
  L.Lx = g.Lx;
  L.Ly = g.Ly;
  L.lx = 0;
  while ((1 << L.lx) < g.nx) ++L.lx;
  L.ly = 0;
  while ((1 << L.ly) < g.ny) ++L.ly;
  L.P = (long long)g.nx * g.ny;
  L.H = g.nx / 2 + 1;
  L.HP = (long long)g.ny * L.H;
  cudaError_t e;
  if ((1 << L.lx) != g.nx || (1 << L.ly) != g.ny) {
    // a side that is not a power of two: the generic kernels (coefficients use parts, sc)
    if ((e = cudaMalloc(&L.parts, sizeof(double) * 5 * kMaxParts))) return e;
    if ((e = cudaMalloc(&L.sc, sizeof(Scal2d)))) return e;
    if ((e = cudaMemset(L.sc, 0, sizeof(Scal2d)))) return e;
    return mr2d_create(L);
  }
  if ((e = cudaMalloc(&L.vec, (size_t)16 * L.HP * 14))) return e;
  if ((e = cudaMalloc(&L.tp, (size_t)16 * L.HP * 4))) return e;
  if ((e = cudaMalloc(&L.coef, sizeof(float) * 6 * L.P))) return e;
  if ((e = cudaMalloc(&L.coef_lo, sizeof(float) * 6 * L.P))) return e;
  if ((e = cudaMalloc(&L.parts, sizeof(double) * 5 * kMaxParts))) return e;
  if ((e = cudaMalloc(&L.sc, sizeof(Scal2d)))) return e;
  if ((e = cudaMalloc(&L.rhs_w, sizeof(double) * 32 * L.P))) return e;
  if ((e = cudaMalloc(&L.stage, sizeof(double) * 7 * L.P))) return e;
  if ((e = cudaMalloc(&L.stage_rec, sizeof(SolveRec) * 2))) return e;
  if ((e = cudaMemset(L.sc, 0, sizeof(Scal2d)))) return e;
  // persistent inner solve
  if ((e = persist2d_grid(L.nx, L.ny, 1, &L.p_grid))) return e;
  L.p_tw = persist2d_tile_width(L.nx, L.ny, 1, L.p_grid);
  const int cu = L.H, ru = L.ny / 2;   // partial-sum slots for the narrowest tiles
  if ((e = cudaMalloc(&L.ehh, sizeof(float) * 3 * L.P))) return e;
  if ((e = cudaMalloc(&L.pinst, sizeof(PInst2d)))) return e;
  if ((e = cudaMalloc(&L.pparts, sizeof(double) * (cu + ru)))) return e;
  if ((e = cudaMalloc(&L.pbar, 2 * sizeof(unsigned)))) return e;
  const PInst2d pi = pinst_of(L);
  if ((e = cudaMemcpy(L.pinst, &pi, sizeof(pi), cudaMemcpyHostToDevice))) return e;
  return cudaSuccess;
}

namespace {

PersistArgs2d persist_args(const Layout2d& L, const void* tw32) {
  PersistArgs2d a;
  a.inst = static_cast<const PInst2d*>(L.pinst);
  a.B = 1;
  a.nx = L.nx;
  a.ny = L.ny;
  a.H = L.H;
  a.lognx = L.lx;
  a.logny = L.ly;
  a.tw = L.p_tw;
  a.maxb = L.p_maxb;
  a.gt = L.p_gt;
  a.col_units = (L.H + L.p_tw - 1) / L.p_tw;
  a.row_units = L.ny / 2;
  a.parts = L.pparts;
  a.bar = L.pbar;
  a.err = reinterpret_cast<int*>(L.pbar + 1);
  a.tw32 = tw32;
  return a;
}

}  // namespace

void layout2d_destroy(Layout2d& L) {
  mr2d_destroy(L);
  if (L.prof) {
    for (auto v : L.prof->a) cudaEventDestroy(v);
    for (auto v : L.prof->b) cudaEventDestroy(v);
    delete L.prof;
    L.prof = nullptr;
  }
  drop_solve_graphs(L);
  cudaFree(L.stage);
  cudaFree(L.stage_rec);
  L.stage = nullptr;
  L.stage_rec = nullptr;
  cudaFree(L.vec);
  cudaFree(L.tp);
  cudaFree(L.coef);
  cudaFree(L.coef_lo);
  cudaFree(L.parts);
  cudaFree(L.sc);
  cudaFree(L.rhs_w);
  cudaFree(L.ehh);
  cudaFree(L.pinst);
  cudaFree(L.pparts);
  cudaFree(L.pbar);
  L.ehh = nullptr;
  L.pinst = nullptr;
  L.pparts = nullptr;
  L.pbar = nullptr;
  L.vec = L.tp = nullptr;
  L.coef = L.coef_lo = nullptr;
  L.parts = nullptr;
  L.sc = nullptr;
  L.rhs_w = nullptr;
}

cudaError_t layout2d_set_inner_form(Layout2d& L, int form, int tile_width) {
  if (L.mr) return cudaErrorNotSupported;            // no persistent form
  if (form == L.inner_form && tile_width == L.p_tw) return cudaSuccess;
  drop_solve_graphs(L);
  L.inner_form = form;
  L.p_tw = tile_width;
  return cudaSuccess;
}

cudaError_t layout2d_set_radix(Layout2d& L, int maxb) {
  if (L.mr || (maxb != 3 && maxb != 4)) return cudaErrorInvalidValue;
  if (maxb == L.p_maxb) return cudaSuccess;
  drop_solve_graphs(L);
  L.p_maxb = maxb;
  return cudaSuccess;
}

cudaError_t layout2d_set_unit_threads(Layout2d& L, int threads) {
  if (L.mr || (threads != 0 && threads != 128 && threads != 256)) return cudaErrorInvalidValue;
  if (threads == L.p_gt) return cudaSuccess;
  drop_solve_graphs(L);
  L.p_gt = threads;
  return cudaSuccess;
}

size_t layout2d_res_bytes(const Layout2d& L) { return (size_t)16 * 2 * (L.HP > 0 ? L.HP : 1); }

// =======================================================================================
// Entry points
// =======================================================================================

cudaError_t launch_grad2d(const Layout2d& L, const void* tw64, const double* f, double* gradf,
                          cudaStream_t s) {
  if (L.mr) return mr2d_grad(L, f, gradf, s);
  // forward transform of f (paired with zero), i k, inverse of both components
  cudaError_t e = rows_r2c<double>(L, tw64, nullptr, f, nullptr, nullptr, nullptr,
                                   tplane(L, 0), tplane(L, 3), nullptr, nullptr, 1, s);
  if (e) return e;
  ColArgs a{};
  a.planes[0] = tplane(L, 0);
  a.K = 1;
  if ((e = cols<double, COL_FWD>(L, tw64, nullptr, a, s))) return e;
  const Modes2d M = modes_of(L);
  k2_spec<double, OP_GRAD><<<grid_for(L.HP, 256), 256, 0, s>>>(
      M, tplane(L, 0), nullptr, tplane(L, 1), tplane(L, 2), nullptr, nullptr, nullptr, nullptr);
  if ((e = cudaGetLastError())) return e;
  return c2r_vec<double>(L, tw64, nullptr, tplane(L, 1), tplane(L, 2), gradf, s);
}

namespace {

// Orszag's 2/3 rule on half planes: modes with |jx| > nx/3 or |jy| > ny/3 set to zero
// (true indices: the Nyquist rows and column are removed too).
__global__ void k2_dealias(Modes2d M, void* p0, void* p1) {
  const long long HP = (long long)M.ny * M.H;
  const double tx = M.nx / 3.0, ty = M.ny / 3.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HP;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)i / M.H, c = (int)i - y * M.H;
    const int ay = y <= (M.ny >> 1) ? y : M.ny - y;
    if (c > tx || ay > ty) {
      st_c<double>(p0, i, mk(0.0, 0.0));
      if (p1) st_c<double>(p1, i, mk(0.0, 0.0));
    }
  }
}

__global__ void k2_sub(long long P, const double* a, const double* b, double* out, double sign) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] + sign * b[i];
}

}  // namespace

cudaError_t launch_dealias2d(const Layout2d& L, const void* tw64, const double* h, double* eta,
                             double* U, double* u, cudaStream_t s) {
  if (L.mr) return cudaErrorNotSupported;
  const Modes2d M = modes_of(L);
  double* zs = L.rhs_w;                        // zeta = eta - h (a free real plane here)
  k2_sub<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, h, zs, -1.0);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  // zeta (paired with zero) through the transform planes
  if ((e = rows_r2c<double>(L, tw64, nullptr, zs, nullptr, nullptr, nullptr, tplane(L, 0),
                            tplane(L, 3), nullptr, nullptr, 1, s)))
    return e;
  ColArgs a{};
  a.planes[0] = tplane(L, 0);
  a.K = 1;
  if ((e = cols<double, COL_FWD>(L, tw64, nullptr, a, s))) return e;
  k2_dealias<<<grid_for(L.HP, 256), 256, 0, s>>>(M, tplane(L, 0), nullptr);
  if ((e = cudaGetLastError())) return e;
  if ((e = cols<double, COL_INV>(L, tw64, nullptr, a, s))) return e;
  if ((e = rows_c2r<double>(L, tw64, nullptr, tplane(L, 0), tplane(L, 3), nullptr, nullptr, zs,
                            nullptr, nullptr, nullptr, 1, s)))
    return e;
  k2_sub<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, h, zs, eta, 1.0);
  if ((e = cudaGetLastError())) return e;
  // the vector fields, two components at a time through the workspace slots
  for (double* v : {U, u}) {
    if (!v) continue;
    if ((e = r2c_vec<double>(L, tw64, nullptr, v, slot(L, 0), slot(L, 1), s))) return e;
    k2_dealias<<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 0), slot(L, 1));
    if ((e = cudaGetLastError())) return e;
    if ((e = c2r_vec<double>(L, tw64, nullptr, slot(L, 0), slot(L, 1), v, s))) return e;
  }
  return cudaSuccess;
}

namespace {

// Pointwise pieces of the 2d non-constraint right-hand side (planes of P doubles).
__global__ void k2_nc_a(long long P, const double* __restrict__ eta, const double* __restrict__ h,
                        const double* __restrict__ u, const double* __restrict__ v,
                        const double* __restrict__ hx, const double* __restrict__ hy,
                        const double* __restrict__ ux, const double* __restrict__ vy,
                        double* __restrict__ d, double* __restrict__ sp, double* __restrict__ z,
                        double* __restrict__ eu, double* __restrict__ ev) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    d[i] = ux[i] + vy[i];
    sp[i] = hx[i] * u[i] + hy[i] * v[i];
    z[i] = eta[i] - h[i];
    eu[i] = eta[i] * u[i];
    ev[i] = eta[i] * v[i];
  }
}

struct NcB {
  const double *eta, *u, *v, *hx, *hy, *ux, *uy, *vx, *vy, *d, *dx, *dy, *sx, *sy, *zx, *zy;
  double *Mx, *My, *Phi;
};

__global__ void k2_nc_b(long long P, double g, NcB a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const double e = a.eta[i], u = a.u[i], v = a.v[i], d = a.d[i];
    const double Q = u * a.dx[i] + v * a.dy[i] - d * d, S = u * a.sx[i] + v * a.sy[i];
    const double Psi = e * e * Q * 0.5 + e * S;
    a.Mx[i] = -e * (u * a.ux[i] + v * a.uy[i]) - g * e * a.zx[i] - a.hx[i] * Psi;
    a.My[i] = -e * (u * a.vx[i] + v * a.vy[i]) - g * e * a.zy[i] - a.hy[i] * Psi;
    a.Phi[i] = e * e * e * Q * (1.0 / 3.0) + e * e * S * 0.5;
  }
}

__global__ void k2_nc_c(long long P, const double* __restrict__ phx, const double* __restrict__ phy,
                        const double* __restrict__ eux, const double* __restrict__ evy,
                        double* __restrict__ Mx, double* __restrict__ My,
                        double* __restrict__ fe) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    Mx[i] += phx[i];
    My[i] += phy[i];
    fe[i] = -(eux[i] + evy[i]);
  }
}

}  // namespace

cudaError_t launch_rhs_nc2d(const Layout2d& L, const void* tw64, double g, const double* eta,
                            const double* u, const double* h, const double* gradh, double* f_eta,
                            double* M, cudaStream_t s) {
  if (L.mr) return cudaErrorNotSupported;
  const long long P = L.P;
  double* w = L.rhs_w;                          // free real planes here
  auto pl = [&](int k) { return w + (long long)k * P; };
  const double* v = u + P;
  const double* hx = gradh;
  const double* hy = gradh + P;
  const int nb = grid_for(P, 256);
  cudaError_t e;
  if ((e = launch_grad2d(L, tw64, u, pl(0), s))) return e;      // u_x, u_y
  if ((e = launch_grad2d(L, tw64, v, pl(2), s))) return e;      // v_x, v_y
  k2_nc_a<<<nb, 256, 0, s>>>(P, eta, h, u, v, hx, hy, pl(0), pl(3), pl(4), pl(5), pl(6), pl(7),
                             pl(8));
  if ((e = cudaGetLastError())) return e;
  if ((e = launch_grad2d(L, tw64, pl(4), pl(9), s))) return e;  // d_x, d_y
  if ((e = launch_grad2d(L, tw64, pl(5), pl(11), s))) return e; // s_x, s_y
  if ((e = launch_grad2d(L, tw64, pl(6), pl(13), s))) return e; // zeta_x, zeta_y
  NcB a{eta, u, v, hx, hy, pl(0), pl(1), pl(2), pl(3), pl(4), pl(9), pl(10), pl(11), pl(12),
        pl(13), pl(14), M, M + P, pl(15)};
  k2_nc_b<<<nb, 256, 0, s>>>(P, g, a);
  if ((e = cudaGetLastError())) return e;
  if ((e = launch_grad2d(L, tw64, pl(15), pl(16), s))) return e;  // Phi_x, Phi_y
  if ((e = launch_grad2d(L, tw64, pl(7), pl(18), s))) return e;   // (eta u)_x
  if ((e = launch_grad2d(L, tw64, pl(8), pl(20), s))) return e;   // (eta v)_y in pl(21)
  k2_nc_c<<<nb, 256, 0, s>>>(P, pl(16), pl(17), pl(18), pl(21), M, M + P, f_eta);
  return cudaGetLastError();
}

cudaError_t launch_coeffs2d(const Layout2d& L, const double* eta, const double* gradh, int kind,
                            SolveRec* rec, cudaStream_t s) {
  k2_coeffs<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, gradh, kind, L.parts, L.sc, rec);
  return cudaGetLastError();
}

cudaError_t launch_apply_G2d(const Layout2d& L, const void* tw64, const double* eta,
                             const double* gradh, const double* u, double* Gu, cudaStream_t s) {
  if (L.mr) return mr2d_apply_G(L, eta, gradh, u, Gu, s);
  k2_coef_planes<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, gradh, L.coef, L.coef_lo, L.ehh);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  if ((e = r2c_vec<double>(L, tw64, nullptr, u, slot(L, 0), slot(L, 1), s))) return e;
  if ((e = matvec<double>(L, tw64, nullptr, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3),
                          nullptr, nullptr, nullptr, nullptr, 0, nullptr, L.sc, 0, 0, nullptr,
                          nullptr, nullptr, nullptr, s)))
    return e;
  return c2r_vec<double>(L, tw64, nullptr, slot(L, 2), slot(L, 3), Gu, s);
}

cudaError_t launch_precond2d(const Layout2d& L, const void* tw64, const SolveRec* rec,
                             const double* r, double* z, cudaStream_t s) {
  if (L.mr) return mr2d_precond(L, rec, r, z, s);
  cudaError_t e = r2c_vec<double>(L, tw64, nullptr, r, slot(L, 0), slot(L, 1), s);
  if (e) return e;
  const Modes2d M = modes_of(L);
  k2_spec<double, OP_AINV><<<grid_for(L.HP, 256), 256, 0, s>>>(
      M, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3), nullptr, nullptr, nullptr, rec);
  if ((e = cudaGetLastError())) return e;
  return c2r_vec<double>(L, tw64, nullptr, slot(L, 2), slot(L, 3), z, s);
}

namespace {

// Inner PCG in precision T on the spectral system G d = r (slots: r 4-5, p 6-7, d 8-9,
// G p 10-11), iterating in chunks with a device-side stop flag.
template <typename T>
cudaError_t inner_pcg(const Layout2d& L, const void* t64, const void* t32, int cap_total,
                      cudaStream_t s) {
  const Modes2d M = modes_of(L);
  const int chunk = 4;
  for (int done_iters = 0;;) {
    for (int c = 0; c < chunk; ++c) {
      cudaError_t e = matvec<T>(L, t64, t32, slot(L, 6), slot(L, 7), slot(L, 10), slot(L, 11),
                                slot(L, 6), slot(L, 7), nullptr, nullptr, 0, nullptr, L.sc, 1, 1,
                                slot(L, 6), slot(L, 7), slot(L, 4), slot(L, 5), s);
      if (e) return e;
      k2_update<T><<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 8), slot(L, 9), slot(L, 4),
                                                        slot(L, 5), slot(L, 6), slot(L, 7),
                                                        slot(L, 10), slot(L, 11), L.sc, L.parts,
                                                        cudaGraphConditionalHandle{}, 0);
      if ((e = cudaGetLastError())) return e;
    }
    done_iters += chunk;
    int done = 0;
    cudaError_t e = cudaMemcpyAsync(&done, &L.sc->done, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    if (done || done_iters > cap_total + chunk) break;
  }
  return cudaSuccess;
}

template <typename T>
__global__ void k2_set_inner(Scal2d* sc, double tol, int cap) {
  sc->tol = tol;
  sc->cap = cap;
  sc->done = 0;
}

__global__ void k2_set_status(Scal2d* sc, int st) { sc->status = st; }

__global__ void k2_reset(Scal2d* sc) {
  sc->iters = 0;
  sc->ticket = 0;
  sc->rz64 = 0.0;
  sc->done = 0;
  sc->refinements = 0;
  sc->it_before = 0;
}

// ---- device-driven solve: the host loop's decisions as one-thread kernels ---------------
// Options of a graph solve, written before the cached graph runs.
__global__ void k2_set_opts(Scal2d* sc, double rtol, double rtol_in, int maxit, int max_refine,
                            int kind) {
  sc->rtol = rtol;
  sc->rtol_in = rtol_in;
  sc->maxit = maxit;
  sc->max_refine = max_refine;
  sc->kind = kind;
}

// Mixed path, after a double-float residual: stop (converged, an error status, a zero
// right-hand side, or out of budget: not converged), or set up the next float32 inner solve
// for G d = r / ||r|| (tolerance as the host loop: 0.3 rtol / ratio within [1e-6, 0.1]).
// Sets the refinement loop's condition; the loop ends within max_refine passes.
__global__ void k2_decide(Scal2d* sc, cudaGraphConditionalHandle hout) {
  unsigned int go = 0u;
  const double bb = sc->bb;
  if (bb > 0.0 && sc->status == SGN_OK) {
    const double ratio = sqrt(fmax(sc->rz64, 0.0)) / sqrt(bb);
    if (ratio > sc->rtol) {
      if (sc->refinements >= sc->max_refine || sc->iters >= sc->maxit) {
        sc->status = SGN_ERR_NOT_CONVERGED;
      } else {
        const double tin =
            sc->rtol_in > 0.0 ? sc->rtol_in : fmin(0.1, fmax(1e-6, 0.3 * sc->rtol / ratio));
        sc->rn = sqrt(sc->rz64);
        sc->tol = tin;
        sc->cap = sc->maxit;
        sc->done = 0;
        sc->it_before = sc->iters;
        go = 1u;
      }
    }
  }
  cudaGraphSetConditional(hout, go);
}

// Mixed path, after an inner solve: a float32 breakdown after some progress keeps the
// correction (the next residual decides); count the pass.
__global__ void k2_after_inner(Scal2d* sc) {
  if (sc->status == SGN_ERR_BREAKDOWN && sc->iters > sc->it_before) sc->status = SGN_OK;
  sc->refinements += 1;
}

// float64 path: one PCG from x0 to sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b).  A zero (or
// non-finite) right-hand side skips the loop (every residual meets the tolerance), and
// k2_finalize returns x = 0.
__global__ void k2_setup_fp64(Scal2d* sc) {
  const double bb = sc->bb;
  sc->tol = bb > 0.0 ? sc->rtol * sqrt(bb) : 1.0e308;
  sc->cap = sc->maxit;
  sc->done = 0;
}

// A zero (or non-finite) right-hand side gives x = 0, as in the host-driven solve.
__global__ void k2_finalize(const Scal2d* sc, double* x, long long n) {
  if (sc->bb > 0.0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

}  // namespace

namespace {

// The solve of launch_pcg2d's host-driven path, with every host decision moved into the
// graph: the refinement loop (mixed) and the inner PCG loop become while nodes whose
// conditions k2_decide, k2_inner_start and k2_update set.  Inputs come from L.stage,
// options from sc (k2_set_opts), the report goes to L.stage_rec[1].
cudaError_t build_solve_graph(const Layout2d& L, const void* tw64, const void* tw32, bool mixed,
                              bool given, cudaGraphExec_t* out, cudaGraph_t* src) {
  const Modes2d M = modes_of(L);
  const long long P = L.P;
  const double* eta = L.stage;
  const double* gh = L.stage + P;
  const double* b = L.stage + 3 * P;
  double* x = L.stage + 5 * P;
  cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaSuccess;
  int capturing = 0;          // streams with a capture begun (ended on every path)
  for (auto& c : cs)
    if (!e) e = cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking);
  if (!e) e = cudaGraphCreate(&g, 0);
  auto begin = [&](int i, cudaGraph_t into) {
    cudaError_t r = cudaStreamBeginCaptureToGraph(cs[i], into, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (!r) capturing |= 1 << i;
    return r;
  };
  auto end = [&](int i) {
    cudaGraph_t dummy;
    capturing &= ~(1 << i);
    cudaError_t r = cudaStreamEndCapture(cs[i], &dummy);
    return r ? r : cudaGetLastError();
  };
  const int blocks = grid_for(L.HP, 256);
  auto inner_loop = [&](auto Tc, cudaStream_t st, cudaGraphConditionalHandle hin) {
    using T = decltype(Tc);
    cudaError_t r = matvec<T>(L, tw64, tw32, slot(L, 6), slot(L, 7), slot(L, 10), slot(L, 11),
                              slot(L, 6), slot(L, 7), nullptr, nullptr, 0, nullptr, L.sc, 1, 1,
                              slot(L, 6), slot(L, 7), slot(L, 4), slot(L, 5), st);
    if (r) return r;
    k2_update<T><<<blocks, 256, 0, st>>>(M, slot(L, 8), slot(L, 9), slot(L, 4), slot(L, 5),
                                         slot(L, 6), slot(L, 7), slot(L, 10), slot(L, 11), L.sc,
                                         L.parts, hin, 1);
    return cudaGetLastError();
  };
  if (!e) e = begin(0, g);
  if (!e) {
    k2_reset<<<1, 1, 0, cs[0]>>>(L.sc);
    if (given) {
      k2_set_given<<<1, 1, 0, cs[0]>>>(L.sc, L.stage_rec);
    } else {
      k2_coeffs<<<grid_for(P, 256), 256, 0, cs[0]>>>(P, eta, gh, -1, L.parts, L.sc, nullptr);
    }
    k2_coef_planes<<<grid_for(P, 256), 256, 0, cs[0]>>>(P, eta, gh, L.coef, L.coef_lo, L.ehh);
    e = cudaGetLastError();
  }
  if (mixed) {
    cudaGraphConditionalHandle hout, hin;
    cudaGraph_t body = nullptr, ibody = nullptr;
    if (!e) e = r2c_vec<df>(L, tw64, tw32, b, slot(L, 0), slot(L, 1), cs[0]);
    if (!e) e = r2c_vec<df>(L, tw64, tw32, x, slot(L, 2), slot(L, 3), cs[0]);
    if (!e) {
      k2_bnorm<df><<<blocks, 256, 0, cs[0]>>>(M, slot(L, 0), slot(L, 1), L.sc, L.parts);
      e = cudaGetLastError();
    }
    // r^ = b^ - G x^ (double-float) into slots 10-11, real-space x on the way
    auto residual = [&](cudaStream_t st) {
      return matvec<df>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 10), slot(L, 11), nullptr,
                        nullptr, slot(L, 0), slot(L, 1), 1, x, L.sc, 0, 0, nullptr, nullptr,
                        nullptr, nullptr, st);
    };
    if (!e) e = residual(cs[0]);
    if (!e) e = cudaGraphConditionalHandleCreate(&hout, g, 0, 0);
    if (!e) {
      k2_decide<<<1, 1, 0, cs[0]>>>(L.sc, hout);
      e = cudaGetLastError();
    }
    if (!e) e = capture_add_while(cs[0], hout, &body);
    // refinement pass: inner solve of G d = r / ||r||, x^ += ||r|| d, next residual, decide
    // the inner solve: one persistent launch, or a while node over the four-kernel iteration
    const bool persist = L.inner_form == 0;
    if (!e) e = begin(1, body);
    if (!e && !persist) e = cudaGraphConditionalHandleCreate(&hin, body, 0, 0);
    if (!e) {
      k2_inner_start<df, float><<<blocks, 256, 0, cs[1]>>>(
          M, slot(L, 10), slot(L, 11), 1.0, slot(L, 4), slot(L, 5), slot(L, 8), slot(L, 9),
          slot(L, 6), slot(L, 7), L.sc, L.parts, 1, persist ? cudaGraphConditionalHandle{} : hin,
          persist ? 0 : 1, L.inner_form == 0 ? 1 : 0);
      e = cudaGetLastError();
    }
    if (persist) {
      if (!e) e = launch_pcg2d_persist(persist_args(L, tw32), L.p_grid, cs[1]);
    } else {
      if (!e) e = capture_add_while(cs[1], hin, &ibody);
      if (!e) e = begin(2, ibody);
      if (!e) e = inner_loop(float(0), cs[2], hin);
      if (!e) e = end(2);
    }
    if (!e) {
      k2_after_inner<<<1, 1, 0, cs[1]>>>(L.sc);
      k2_accumulate<df, float><<<blocks, 256, 0, cs[1]>>>(M, slot(L, 2), slot(L, 3), slot(L, 8),
                                                         slot(L, 9), 1.0, L.sc,
                                                         L.inner_form == 0 ? 1 : 0);
      e = cudaGetLastError();
    }
    if (!e) e = residual(cs[1]);
    if (!e) {
      k2_decide<<<1, 1, 0, cs[1]>>>(L.sc, hout);
      e = cudaGetLastError();
    }
    if (!e) e = end(1);
  } else {
    cudaGraphConditionalHandle hin;
    cudaGraph_t ibody = nullptr;
    if (!e) e = r2c_vec<double>(L, tw64, tw32, b, slot(L, 0), slot(L, 1), cs[0]);
    if (!e) e = r2c_vec<double>(L, tw64, tw32, x, slot(L, 2), slot(L, 3), cs[0]);
    if (!e) {
      k2_bnorm<double><<<blocks, 256, 0, cs[0]>>>(M, slot(L, 0), slot(L, 1), L.sc, L.parts);
      e = cudaGetLastError();
    }
    // r = b - G x0 (slots 4-5), then PCG in float64 with the correction in slots 8-9
    if (!e) e = matvec<double>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 4), slot(L, 5),
                               nullptr, nullptr, slot(L, 0), slot(L, 1), 1, nullptr, L.sc, 0, 0,
                               nullptr, nullptr, nullptr, nullptr, cs[0]);
    if (!e) e = cudaGraphConditionalHandleCreate(&hin, g, 0, 0);
    if (!e) {
      k2_setup_fp64<<<1, 1, 0, cs[0]>>>(L.sc);
      k2_inner_start<double, double><<<blocks, 256, 0, cs[0]>>>(
          M, slot(L, 4), slot(L, 5), 1.0, slot(L, 12), slot(L, 13), slot(L, 8), slot(L, 9),
          slot(L, 6), slot(L, 7), L.sc, L.parts, 0, hin, 1, 0);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(slot(L, 4), slot(L, 12), (size_t)16 * L.HP,
                                cudaMemcpyDeviceToDevice, cs[0]);
    if (!e) e = cudaMemcpyAsync(slot(L, 5), slot(L, 13), (size_t)16 * L.HP,
                                cudaMemcpyDeviceToDevice, cs[0]);
    if (!e) e = capture_add_while(cs[0], hin, &ibody);
    if (!e) e = begin(1, ibody);
    if (!e) e = inner_loop(double(0), cs[1], hin);
    if (!e) e = end(1);
    if (!e) {
      k2_accumulate<double, double><<<blocks, 256, 0, cs[0]>>>(M, slot(L, 2), slot(L, 3),
                                                               slot(L, 8), slot(L, 9), 1.0,
                                                               nullptr, 0);
      e = cudaGetLastError();
    }
    // final float64 residual for the report and x = F^{-1} x^
    if (!e) e = matvec<double>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 10), slot(L, 11),
                               nullptr, nullptr, slot(L, 0), slot(L, 1), 1, x, L.sc, 0, 0,
                               nullptr, nullptr, nullptr, nullptr, cs[0]);
  }
  if (!e) {
    k2_finalize<<<grid_for(2 * P, 256), 256, 0, cs[0]>>>(L.sc, x, 2 * P);
    k2_report<<<1, 1, 0, cs[0]>>>(L.sc, L.stage_rec + 1, -1);
    e = cudaGetLastError();
  }
  if (!e) e = end(0);
  for (int i = 2; i >= 0; --i)
    if (capturing & (1 << i)) end(i);          // a failed build: close its captures
  if (!e) e = cudaGraphInstantiate(out, g, 0);
  for (auto& c : cs)
    if (c) cudaStreamDestroy(c);
  // the source graph lives as long as its executable graph (both go in drop_solve_graphs).
  // A graph whose build failed is left alone: destroying one whose capture into a
  // conditional node's body had failed crashed the driver.  The layout then solves on the
  // host-driven path, so this happens at most once per layout.
  if (!e) *src = g;
  return e;
}

}  // namespace

cudaError_t launch_pcg2d(const Layout2d& L, const void* tw64, const void* tw32, int precision,
                         const double* eta, const double* gradh, const double* b, double* x,
                         const SolveRec* given, int kind, double rtol, double rtol_inner,
                         int maxit, int max_refine, SolveRec* rec, cudaStream_t s) {
  if (L.mr)
    return mr2d_pcg(L, precision, eta, gradh, b, x, given, kind, rtol, rtol_inner, maxit,
                    max_refine, rec, s);
  const Modes2d M = modes_of(L);
  cudaError_t e;
  // ---- device-driven: one graph launch between staging copies
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (!L.solve_graph_off && !L.prof && cudaStreamIsCapturing(s, &cst) == cudaSuccess &&
      cst == cudaStreamCaptureStatusNone) {
    const int mi = precision == SGN_PREC_MIXED ? 1 : 0, gi = given ? 1 : 0;
    cudaGraphExec_t& ex = L.solve_exec[mi][gi];
    if (!ex && build_solve_graph(L, tw64, tw32, mi == 1, gi == 1, &ex,
                                 &L.solve_graph[mi][gi]) != cudaSuccess) {
      cudaGetLastError();
      ex = nullptr;
      L.solve_graph_off = true;
    }
    if (ex) {
      const long long P = L.P;
      const size_t d = sizeof(double);
      if ((e = cudaMemcpyAsync(L.stage, eta, d * P, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + P, gradh, d * 2 * P, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + 3 * P, b, d * 2 * P, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(L.stage + 5 * P, x, d * 2 * P, cudaMemcpyDeviceToDevice, s)))
        return e;
      if (given && (e = cudaMemcpyAsync(L.stage_rec, given, sizeof(SolveRec),
                                        cudaMemcpyDeviceToDevice, s)))
        return e;
      k2_set_opts<<<1, 1, 0, s>>>(L.sc, rtol, rtol_inner, maxit, max_refine, kind);
      if ((e = cudaGetLastError()) || (e = cudaGraphLaunch(ex, s))) return e;
      if ((e = cudaMemcpyAsync(x, L.stage + 5 * P, d * 2 * P, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemcpyAsync(rec, L.stage_rec + 1, sizeof(SolveRec), cudaMemcpyDeviceToDevice,
                               s)))
        return e;
      return cudaSuccess;
    }
  }
  // ---- host-driven
  k2_reset<<<1, 1, 0, s>>>(L.sc);
  if (given) {
    k2_set_given<<<1, 1, 0, s>>>(L.sc, given);
  } else {
    k2_coeffs<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, gradh, kind, L.parts, L.sc, nullptr);
  }
  k2_coef_planes<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, gradh, L.coef, L.coef_lo, L.ehh);
  if ((e = cudaGetLastError())) return e;
  Scal2d h{};
  if ((e = cudaMemcpyAsync(&h, L.sc, sizeof(Scal2d), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  if (h.status != SGN_OK) {
    k2_report<<<1, 1, 0, s>>>(L.sc, rec, 0);
    return cudaGetLastError();
  }
  const bool mixed = precision == SGN_PREC_MIXED;
  // b^ -> slots 0-1, x0^ -> slots 2-3 (high precision)
  if (mixed) {
    if ((e = r2c_vec<df>(L, tw64, tw32, b, slot(L, 0), slot(L, 1), s))) return e;
    if ((e = r2c_vec<df>(L, tw64, tw32, x, slot(L, 2), slot(L, 3), s))) return e;
    k2_bnorm<df><<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 0), slot(L, 1), L.sc, L.parts);
  } else {
    if ((e = r2c_vec<double>(L, tw64, tw32, b, slot(L, 0), slot(L, 1), s))) return e;
    if ((e = r2c_vec<double>(L, tw64, tw32, x, slot(L, 2), slot(L, 3), s))) return e;
    k2_bnorm<double><<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 0), slot(L, 1), L.sc,
                                                         L.parts);
  }
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(&h, L.sc, sizeof(Scal2d), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  const double bnorm = sqrt(fmax(h.bb, 0.0));
  if (!(bnorm > 0.0)) {
    cudaMemsetAsync(x, 0, sizeof(double) * 2 * L.P, s);
    k2_report<<<1, 1, 0, s>>>(L.sc, rec, 0);
    return cudaGetLastError();
  }
  if (!mixed) {
    // r = b - G x0 (slots 4-5), then PCG in float64 with x^ accumulating in slots 2-3
    if ((e = matvec<double>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 4), slot(L, 5),
                            nullptr, nullptr, slot(L, 0), slot(L, 1), 1, nullptr, L.sc, 0, 0,
                            nullptr, nullptr, nullptr, nullptr, s)))
      return e;
    // start: copy r into the T slots (scale 1), x -> separate accumulation in slots 8-9
    k2_set_inner<double><<<1, 1, 0, s>>>(L.sc, rtol * bnorm, maxit);
    k2_inner_start<double, double><<<grid_for(L.HP, 256), 256, 0, s>>>(
        M, slot(L, 4), slot(L, 5), 1.0, slot(L, 12), slot(L, 13), slot(L, 8), slot(L, 9),
        slot(L, 6), slot(L, 7), L.sc, L.parts, 0, cudaGraphConditionalHandle{}, 0, 0);
    if ((e = cudaGetLastError())) return e;
    // move r into slots 4-5 for the loop
    cudaMemcpyAsync(slot(L, 4), slot(L, 12), (size_t)16 * L.HP, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(slot(L, 5), slot(L, 13), (size_t)16 * L.HP, cudaMemcpyDeviceToDevice, s);
    if ((e = inner_pcg<double>(L, tw64, tw32, maxit, s))) return e;
    k2_accumulate<double, double><<<grid_for(L.HP, 256), 256, 0, s>>>(
        M, slot(L, 2), slot(L, 3), slot(L, 8), slot(L, 9), 1.0, nullptr, 0);
    // final float64 residual for the report and x = F^{-1} x^
    if ((e = matvec<double>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 10), slot(L, 11),
                            nullptr, nullptr, slot(L, 0), slot(L, 1), 1, x, L.sc, 0, 0, nullptr,
                            nullptr, nullptr, nullptr, s)))
      return e;
    k2_report<<<1, 1, 0, s>>>(L.sc, rec, 0);
    return cudaGetLastError();
  }
  // mixed: double-float refinement around float32 inner solves
  int refinements = 0;
  for (;;) {
    // r^ = b^ - G x^ (double-float) into slots 10-11 (as df), writes real-space x
    if ((e = matvec<df>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 10), slot(L, 11), nullptr,
                        nullptr, slot(L, 0), slot(L, 1), 1, x, L.sc, 0, 0, nullptr, nullptr,
                        nullptr, nullptr, s)))
      return e;
    if ((e = cudaMemcpyAsync(&h, L.sc, sizeof(Scal2d), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    const double ratio = sqrt(fmax(h.rz64, 0.0)) / bnorm;
    if (ratio <= rtol || h.status != SGN_OK) break;
    if (refinements >= max_refine || h.iters >= maxit) {
      k2_set_status<<<1, 1, 0, s>>>(L.sc, SGN_ERR_NOT_CONVERGED);
      k2_report<<<1, 1, 0, s>>>(L.sc, rec, refinements);
      return cudaGetLastError();
    }
    const double rn = sqrt(h.rz64);
    const double tin =
        rtol_inner > 0.0 ? rtol_inner : fmin(0.1, fmax(1e-6, 0.3 * rtol / ratio));
    k2_set_inner<float><<<1, 1, 0, s>>>(L.sc, tin, maxit);
    k2_inner_start<df, float><<<grid_for(L.HP, 256), 256, 0, s>>>(
        M, slot(L, 10), slot(L, 11), 1.0 / rn, slot(L, 4), slot(L, 5), slot(L, 8), slot(L, 9),
        slot(L, 6), slot(L, 7), L.sc, L.parts, 0, cudaGraphConditionalHandle{}, 0,
        L.inner_form == 0 ? 1 : 0);
    if ((e = cudaGetLastError())) return e;
    const int it_before = h.iters;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (L.prof && L.inner_form == 0) {
      for (auto& v : ev)
        if ((e = cudaEventCreate(&v))) return e;
      cudaEventRecord(ev[0], s);
    }
    if ((e = L.inner_form == 0 ? launch_pcg2d_persist(persist_args(L, tw32), L.p_grid, s)
                               : inner_pcg<float>(L, tw64, tw32, maxit, s)))
      return e;
    if (ev[1]) cudaEventRecord(ev[1], s);
    {
      // a float32 breakdown after some progress keeps the correction (see the 1d solve)
      Scal2d hs{};
      if ((e = cudaMemcpyAsync(&hs, L.sc, sizeof(Scal2d), cudaMemcpyDeviceToHost, s))) return e;
      if ((e = cudaStreamSynchronize(s))) return e;
      if (hs.status == SGN_ERR_BREAKDOWN && hs.iters > it_before)
        k2_set_status<<<1, 1, 0, s>>>(L.sc, SGN_OK);
      if (ev[1]) {
        L.prof->a.push_back(ev[0]);
        L.prof->b.push_back(ev[1]);
        L.prof->iters.push_back(hs.iters - it_before);
      }
    }
    k2_accumulate<df, float><<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 2), slot(L, 3),
                                                                  slot(L, 8), slot(L, 9), rn,
                                                                  nullptr,
                                                                  L.inner_form == 0 ? 1 : 0);
    if ((e = cudaGetLastError())) return e;
    ++refinements;
  }
  k2_report<<<1, 1, 0, s>>>(L.sc, rec, refinements);
  return cudaGetLastError();
}

// =======================================================================================
// Batches of 2d instances on one grid
// =======================================================================================

cudaError_t batch2d_create(Batch2d& Bt, Layout2d& first, const sgn_grid& g, int B) {
  Bt.B = B;
  Bt.more.resize(B - 1);
  cudaError_t e;
  for (auto& L : Bt.more)
    if ((e = layout2d_create(L, g))) return e;
  const long long P = first.P;
  if ((e = cudaMalloc(&Bt.stage, sizeof(double) * 7 * P * B))) return e;
  if ((e = persist2d_grid(first.nx, first.ny, B, &Bt.p_grid))) return e;
  Bt.p_tw = persist2d_tile_width(first.nx, first.ny, B, Bt.p_grid);
  if ((e = cudaMalloc(&Bt.pinst, sizeof(PInst2d) * B))) return e;
  if ((e = cudaMalloc(&Bt.pparts, sizeof(double) * B * (first.H + first.ny / 2)))) return e;
  if ((e = cudaMalloc(&Bt.pbar, 2 * sizeof(unsigned)))) return e;
  std::vector<PInst2d> pi(B);
  for (int b = 0; b < B; ++b) pi[b] = pinst_of(Bt.inst(first, b));
  return cudaMemcpy(Bt.pinst, pi.data(), sizeof(PInst2d) * B, cudaMemcpyHostToDevice);
}

void batch2d_destroy(Batch2d& Bt) {
  for (auto& L : Bt.more) layout2d_destroy(L);
  Bt.more.clear();
  cudaFree(Bt.stage);
  cudaFree(Bt.pinst);
  cudaFree(Bt.pparts);
  cudaFree(Bt.pbar);
  Bt.stage = nullptr;
  Bt.pinst = nullptr;
  Bt.pparts = nullptr;
  Bt.pbar = nullptr;
  Bt.B = 0;
}

cudaError_t batch2d_stage_in(const Layout2d& L, double* st, int b, long long Ptot,
                             const double* scal, const double* vec0, const double* vec1,
                             const double* vec2, cudaStream_t s) {
  const long long P = L.P;
  const size_t n = sizeof(double) * P;
  cudaError_t e;
  if (scal && (e = cudaMemcpyAsync(st, scal + b * P, n, cudaMemcpyDeviceToDevice, s))) return e;
  const double* v[3] = {vec0, vec1, vec2};
  for (int q = 0; q < 3; ++q) {
    if (!v[q]) continue;
    double* d = st + (1 + 2 * q) * P;
    if ((e = cudaMemcpyAsync(d, v[q] + b * P, n, cudaMemcpyDeviceToDevice, s)) ||
        (e = cudaMemcpyAsync(d + P, v[q] + Ptot + b * P, n, cudaMemcpyDeviceToDevice, s)))
      return e;
  }
  return cudaSuccess;
}

cudaError_t batch2d_stage_out(const Layout2d& L, const double* stvec, int b, long long Ptot,
                              double* vec, cudaStream_t s) {
  const long long P = L.P;
  const size_t n = sizeof(double) * P;
  cudaError_t e = cudaMemcpyAsync(vec + b * P, stvec, n, cudaMemcpyDeviceToDevice, s);
  if (e) return e;
  return cudaMemcpyAsync(vec + Ptot + b * P, stvec + P, n, cudaMemcpyDeviceToDevice, s);
}

namespace {
__global__ void k2_mark_done(Scal2d* sc) { sc->done = 1; }
}  // namespace

cudaError_t launch_pcg2d_batch(Layout2d& first, Batch2d& Bt, const void* tw64, const void* tw32,
                               int precision, const double* eta, const double* gradh,
                               const double* b, double* x, const SolveRec* given, int kind,
                               double rtol, double rtol_inner, int maxit, int max_refine,
                               SolveRec* rec, cudaStream_t s) {
  const int B = Bt.B;
  const long long P = first.P, Ptot = P * B;
  cudaError_t e;
  auto st_of = [&](int i) { return Bt.stage + 7 * P * i; };
  for (int i = 0; i < B; ++i)
    if ((e = batch2d_stage_in(first, st_of(i), i, Ptot, eta, gradh, b, x, s))) return e;
  if (precision != SGN_PREC_MIXED) {
    // float64: each instance through the single-instance solve
    for (int i = 0; i < B; ++i) {
      double* st = st_of(i);
      if ((e = launch_pcg2d(Bt.inst(first, i), tw64, tw32, precision, st, st + P, st + 3 * P,
                            st + 5 * P, given ? given + i : nullptr, kind, rtol, rtol_inner,
                            maxit, max_refine, rec + i, s)) ||
          (e = batch2d_stage_out(first, st + 5 * P, i, Ptot, x, s)))
        return e;
    }
    return cudaSuccess;
  }
  // mixed: double-float refinement of every instance around one persistent launch per pass
  std::vector<Scal2d> h(B);
  auto fetch = [&]() {
    for (int i = 0; i < B; ++i) {
      cudaError_t r = cudaMemcpyAsync(&h[i], Bt.inst(first, i).sc, sizeof(Scal2d),
                                      cudaMemcpyDeviceToHost, s);
      if (r) return r;
    }
    return cudaStreamSynchronize(s);
  };
  for (int i = 0; i < B; ++i) {
    Layout2d& L = Bt.inst(first, i);
    const Modes2d M = modes_of(L);
    const double* st = st_of(i);
    k2_reset<<<1, 1, 0, s>>>(L.sc);
    if (given) {
      k2_set_given<<<1, 1, 0, s>>>(L.sc, given + i);
    } else {
      k2_coeffs<<<grid_for(P, 256), 256, 0, s>>>(P, st, st + P, kind, L.parts, L.sc, nullptr);
    }
    k2_coef_planes<<<grid_for(P, 256), 256, 0, s>>>(P, st, st + P, L.coef, L.coef_lo, L.ehh);
    if ((e = cudaGetLastError()) ||
        (e = r2c_vec<df>(L, tw64, tw32, st + 3 * P, slot(L, 0), slot(L, 1), s)) ||
        (e = r2c_vec<df>(L, tw64, tw32, st + 5 * P, slot(L, 2), slot(L, 3), s)))
      return e;
    k2_bnorm<df><<<grid_for(L.HP, 256), 256, 0, s>>>(M, slot(L, 0), slot(L, 1), L.sc, L.parts);
    if ((e = cudaGetLastError())) return e;
  }
  if ((e = fetch())) return e;
  // per instance: 0 refining, 1 finished
  std::vector<int> fin(B, 0), refinements(B, 0), it_before(B, 0), pass(B, 0);
  std::vector<double> bnorm(B, 0.0), rn(B, 0.0);
  for (int i = 0; i < B; ++i) {
    bnorm[i] = sqrt(fmax(h[i].bb, 0.0));
    if (h[i].status != SGN_OK) {
      fin[i] = 1;
    } else if (!(bnorm[i] > 0.0)) {
      if ((e = cudaMemsetAsync(st_of(i) + 5 * P, 0, sizeof(double) * 2 * P, s))) return e;
      fin[i] = 1;
    }
  }
  const PersistArgs2d pa = [&] {
    PersistArgs2d a;
    a.inst = static_cast<const PInst2d*>(Bt.pinst);
    a.B = B;
    a.nx = first.nx;
    a.ny = first.ny;
    a.H = first.H;
    a.lognx = first.lx;
    a.logny = first.ly;
    a.tw = Bt.p_tw;
    a.maxb = first.p_maxb;
    a.gt = first.p_gt;
    a.col_units = (first.H + Bt.p_tw - 1) / Bt.p_tw;
    a.row_units = first.ny / 2;
    a.parts = Bt.pparts;
    a.bar = Bt.pbar;
    a.err = reinterpret_cast<int*>(Bt.pbar + 1);
    a.tw32 = tw32;
    return a;
  }();
  for (;;) {
    for (int i = 0; i < B; ++i) {
      if (fin[i]) continue;
      Layout2d& L = Bt.inst(first, i);
      if ((e = matvec<df>(L, tw64, tw32, slot(L, 2), slot(L, 3), slot(L, 10), slot(L, 11),
                          nullptr, nullptr, slot(L, 0), slot(L, 1), 1, st_of(i) + 5 * P, L.sc,
                          0, 0, nullptr, nullptr, nullptr, nullptr, s)))
        return e;
    }
    if ((e = fetch())) return e;
    bool any = false;
    for (int i = 0; i < B; ++i) {
      Layout2d& L = Bt.inst(first, i);
      pass[i] = 0;
      if (!fin[i]) {
        const double ratio = sqrt(fmax(h[i].rz64, 0.0)) / bnorm[i];
        if (ratio <= rtol || h[i].status != SGN_OK) {
          fin[i] = 1;
        } else if (refinements[i] >= max_refine || h[i].iters >= maxit) {
          k2_set_status<<<1, 1, 0, s>>>(L.sc, SGN_ERR_NOT_CONVERGED);
          fin[i] = 1;
        } else {
          const Modes2d M = modes_of(L);
          rn[i] = sqrt(h[i].rz64);
          const double tin =
              rtol_inner > 0.0 ? rtol_inner : fmin(0.1, fmax(1e-6, 0.3 * rtol / ratio));
          k2_set_inner<float><<<1, 1, 0, s>>>(L.sc, tin, maxit);
          k2_inner_start<df, float><<<grid_for(L.HP, 256), 256, 0, s>>>(
              M, slot(L, 10), slot(L, 11), 1.0 / rn[i], slot(L, 4), slot(L, 5), slot(L, 8),
              slot(L, 9), slot(L, 6), slot(L, 7), L.sc, L.parts, 0, cudaGraphConditionalHandle{},
              0, 1);     // a batch always runs the persistent inner solve
          it_before[i] = h[i].iters;
          pass[i] = 1;
          any = true;
        }
      }
      if (!pass[i]) k2_mark_done<<<1, 1, 0, s>>>(L.sc);
    }
    if ((e = cudaGetLastError())) return e;
    if (!any) break;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (first.prof) {
      for (auto& v : ev)
        if ((e = cudaEventCreate(&v))) return e;
      cudaEventRecord(ev[0], s);
    }
    if ((e = launch_pcg2d_persist(pa, Bt.p_grid, s))) return e;
    if (ev[1]) cudaEventRecord(ev[1], s);
    if ((e = fetch())) return e;
    long long its = 0;
    for (int i = 0; i < B; ++i) {
      if (!pass[i]) continue;
      Layout2d& L = Bt.inst(first, i);
      its += h[i].iters - it_before[i];
      // a float32 breakdown after some progress keeps the correction (see the 1d solve)
      if (h[i].status == SGN_ERR_BREAKDOWN && h[i].iters > it_before[i])
        k2_set_status<<<1, 1, 0, s>>>(L.sc, SGN_OK);
      k2_accumulate<df, float><<<grid_for(L.HP, 256), 256, 0, s>>>(
          modes_of(L), slot(L, 2), slot(L, 3), slot(L, 8), slot(L, 9), rn[i], nullptr, 1);
      ++refinements[i];
    }
    if ((e = cudaGetLastError())) return e;
    if (ev[1]) {
      first.prof->a.push_back(ev[0]);
      first.prof->b.push_back(ev[1]);
      first.prof->iters.push_back(its);
    }
  }
  for (int i = 0; i < B; ++i) {
    k2_report<<<1, 1, 0, s>>>(Bt.inst(first, i).sc, rec + i, refinements[i]);
    if ((e = batch2d_stage_out(first, st_of(i) + 5 * P, i, Ptot, x, s))) return e;
  }
  return cudaGetLastError();
}

namespace {

// Right-hand side (Def:bigF) in four transform passes (see k2_rhs_stage for plane indices):
// div u, div(eta u) and grad(div u) from one pass of (u, v, eta u, eta v); grad zeta and
// grad s; the two components of div(eta u (x) u); grad Phi.  Sums of derivatives are formed
// in spectral space, so only the twelve planes the pointwise stages read are transformed
// back.  The transforms run in T (float64, or double-float for the mixed path); the
// pointwise stages and the intermediate planes are float64.
template <typename T>
cudaError_t rhs2d(const Layout2d& L, const void* tw64, const void* tw32, double g,
                  const double* eta, const double* u, const double* h, const double* gradh,
                  double* f_eta, double* f_U, cudaStream_t s) {
  double* w = L.rhs_w;
  const long long P = L.P;
  auto W = [&](int q) { return w + (long long)q * P; };
  const int gb = grid_for(P, 256);
  cudaError_t e;
  auto grad_pair = [&](const double* a, const double* b, double* ax, double* ay, double* bx,
                       double* by) -> cudaError_t {
    cudaError_t r = rows_r2c<T>(L, tw64, tw32, a, b, nullptr, nullptr, tplane(L, 0),
                                     tplane(L, 1), nullptr, nullptr, 1, s);
    if (r) return r;
    ColArgs c{};
    c.planes[0] = tplane(L, 0);
    c.planes[1] = tplane(L, 1);
    c.K = 2;
    if ((r = cols<T, COL_FWD>(L, tw64, tw32, c, s))) return r;
    const Modes2d M = modes_of(L);
    k2_spec<T, OP_GRAD><<<grid_for(L.HP, 256), 256, 0, s>>>(
        M, tplane(L, 0), tplane(L, 1), slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3), nullptr,
        nullptr);
    if ((r = cudaGetLastError())) return r;
    ColArgs ci{};
    ci.planes[0] = slot(L, 0);
    ci.planes[1] = slot(L, 1);
    ci.planes[2] = slot(L, 2);
    ci.planes[3] = slot(L, 3);
    ci.K = 4;
    if ((r = cols<T, COL_INV>(L, tw64, tw32, ci, s))) return r;
    return rows_c2r<T>(L, tw64, tw32, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3), ax,
                            ay, bx, by, 2, s);
  };
  // Pass of four real fields through the forward transform, a spectral combination and the
  // inverse transform of nout planes (written to out[0..nout) as real planes).
  auto combo = [&](const double* a, const double* b, const double* c, const double* d, int K,
                   int mode, int nout, double* const* out) -> cudaError_t {
    cudaError_t r = rows_r2c<T>(L, tw64, tw32, a, b, c, d, tplane(L, 0), tplane(L, 1),
                                tplane(L, 2), tplane(L, 3), (K + 1) / 2, s);
    if (r) return r;
    ColArgs cf{};
    for (int q = 0; q < 4; ++q) cf.planes[q] = tplane(L, q);
    cf.K = K;
    if ((r = cols<T, COL_FWD>(L, tw64, tw32, cf, s))) return r;
    const Modes2d M = modes_of(L);
    if (mode == RHS_DIVD)
      k2_spec_rhs<T, RHS_DIVD><<<grid_for(L.HP, 256), 256, 0, s>>>(
          M, tplane(L, 0), tplane(L, 1), tplane(L, 2), tplane(L, 3), slot(L, 0), slot(L, 1),
          slot(L, 2), slot(L, 3));
    else
      k2_spec_rhs<T, RHS_DIV2><<<grid_for(L.HP, 256), 256, 0, s>>>(
          M, tplane(L, 0), tplane(L, 1), tplane(L, 2), nullptr, slot(L, 0), slot(L, 1), nullptr,
          nullptr);
    if ((r = cudaGetLastError())) return r;
    ColArgs ci{};
    for (int q = 0; q < 4; ++q) ci.planes[q] = slot(L, q);
    ci.K = nout;
    if ((r = cols<T, COL_INV>(L, tw64, tw32, ci, s))) return r;
    return rows_c2r<T>(L, tw64, tw32, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3), out[0],
                       out[1], nout > 2 ? out[2] : nullptr, nout > 2 ? out[3] : nullptr,
                       nout / 2, s);
  };
  k2_rhs_stage<double><<<gb, 256, 0, s>>>(0, P, g, eta, u, h, gradh, w, f_eta, f_U);
  if ((e = cudaGetLastError())) return e;
  // d = div u, m = div(eta u), grad d from one pass of (u, v, eta u, eta v)
  {
    double* out[4] = {W(7), W(14), W(22), W(23)};
    if ((e = combo(u, u + P, W(0), W(1), 4, RHS_DIVD, 4, out))) return e;
  }
  if ((e = grad_pair(W(2), W(3), W(18), W(19), W(20), W(21)))) return e;   // grad zeta, grad s
  // div(eta u (x) u) from (eta u u, eta u v, eta v v)
  {
    double* out[4] = {W(24), W(26), nullptr, nullptr};
    if ((e = combo(W(4), W(5), W(6), nullptr, 3, RHS_DIV2, 2, out))) return e;
  }
  k2_rhs_stage<double><<<gb, 256, 0, s>>>(2, P, g, eta, u, h, gradh, w, f_eta, f_U);
  if ((e = cudaGetLastError())) return e;
  if ((e = grad_pair(W(8), nullptr, W(30), W(31), nullptr, nullptr))) return e;
  k2_rhs_stage<double><<<gb, 256, 0, s>>>(3, P, g, eta, u, h, gradh, w, f_eta, f_U);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rhs2d(const Layout2d& L, const void* tw64, const void* tw32, int precision,
                         double g, const double* eta, const double* u, const double* h,
                         const double* gradh, double* f_eta, double* f_U, cudaStream_t s) {
  if (L.mr) return mr2d_rhs(L, g, eta, u, h, gradh, f_eta, f_U, s);
  return precision == SGN_PREC_MIXED
             ? rhs2d<df>(L, tw64, tw32, g, eta, u, h, gradh, f_eta, f_U, s)
             : rhs2d<double>(L, tw64, tw32, g, eta, u, h, gradh, f_eta, f_U, s);
}

cudaError_t launch_lincomb2d(const Layout2d& L, const double* dt, double* out,
                             const double* const* x, const double* a, int nx,
                             const double* const* f, const double* c, int nf, int components,
                             cudaStream_t s) {
  const long long n = L.P * components;
  const double* X[4] = {nullptr, nullptr, nullptr, nullptr};
  const double* F[4] = {nullptr, nullptr, nullptr, nullptr};
  double A[4] = {0, 0, 0, 0}, Cc[4] = {0, 0, 0, 0};
  for (int t = 0; t < nx; ++t) {
    X[t] = x[t];
    A[t] = a[t];
  }
  for (int t = 0; t < nf; ++t) {
    F[t] = f[t];
    Cc[t] = c[t];
  }
  k2_lincomb<<<grid_for(n, 256), 256, 0, s>>>(n, out, X[0], X[1], X[2], X[3], A[0], A[1], A[2],
                                               A[3], nx, F[0], F[1], F[2], F[3], Cc[0], Cc[1],
                                               Cc[2], Cc[3], nf, dt);
  return cudaGetLastError();
}

cudaError_t launch_linimp_res2d(const Layout2d& L, const void* tw64, const SolveRec* A,
                                const double* eta, const double* gradh, const double* u,
                                const double* U, void* res_hat, cudaStream_t s) {
  if (L.mr) return cudaErrorNotSupported;
  // res^ = A u^ - (G u)^ + U^, float64, stored as two half planes in res_hat
  k2_coef_planes<<<grid_for(L.P, 256), 256, 0, s>>>(L.P, eta, gradh, L.coef, L.coef_lo, L.ehh);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  if ((e = r2c_vec<double>(L, tw64, nullptr, u, slot(L, 0), slot(L, 1), s))) return e;
  if ((e = r2c_vec<double>(L, tw64, nullptr, U, slot(L, 4), slot(L, 5), s))) return e;
  if ((e = matvec<double>(L, tw64, nullptr, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3),
                          nullptr, nullptr, nullptr, nullptr, 0, nullptr, L.sc, 0, 0, nullptr,
                          nullptr, nullptr, nullptr, s)))
    return e;
  char* r = static_cast<char*>(res_hat);
  const Modes2d M = modes_of(L);
  k2_linimp_combine<double><<<grid_for(L.HP, 256), 256, 0, s>>>(
      M, A, slot(L, 0), slot(L, 1), slot(L, 2), slot(L, 3), slot(L, 4), slot(L, 5), r,
      r + (size_t)16 * L.HP);
  return cudaGetLastError();
}

cudaError_t launch_linimp_solve2d(const Layout2d& L, const void* tw64, const SolveRec* A,
                                  const void* res1_hat, const void* res0_hat, double c1,
                                  double c0, double* u, cudaStream_t s) {
  if (L.mr) return cudaErrorNotSupported;
  const char* r1 = static_cast<const char*>(res1_hat);
  const char* r0 = static_cast<const char*>(res0_hat);
  const size_t off = (size_t)16 * L.HP;
  k2_axpby<double><<<grid_for(L.HP, 256), 256, 0, s>>>(L.HP, slot(L, 4), slot(L, 5), r1,
                                                        r1 + off, r0, r0 + off, c1, c0);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  const Modes2d M = modes_of(L);
  k2_spec<double, OP_AINV><<<grid_for(L.HP, 256), 256, 0, s>>>(
      M, slot(L, 4), slot(L, 5), slot(L, 6), slot(L, 7), nullptr, nullptr, nullptr, A);
  if ((e = cudaGetLastError())) return e;
  return c2r_vec<double>(L, tw64, nullptr, slot(L, 6), slot(L, 7), u, s);
}

}  // namespace sgn
