// Launchers of the register-FFT 1d kernels: one launch per size class.  The kernels
// (sgn_1d_pcg.cuh: a5/a6 solve, sgn_1d_rhs.cuh: a7 right-hand side) are instantiated per
// size in the sgn_1d_l*.cu translation units, which compile in parallel.
#include "sgn_1d_pcg.cuh"
#include "sgn_1d_rhs.cuh"

namespace sgn {

extern template cudaError_t pcg1d_launch<3, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<4, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<5, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<6, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<7, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<8, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<9, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<10, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<11, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<12, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<13, 1>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<12, 2>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<13, 2>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t pcg1d_launch<14, 2>(const PcgArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<3, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<4, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<5, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<6, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<7, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<8, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<9, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<10, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<11, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<12, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<13, 1>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<12, 2>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<13, 2>(const RhsArgs&, int, int, cudaStream_t);
extern template cudaError_t rhs1d_launch<14, 2>(const RhsArgs&, int, int, cudaStream_t);

namespace {

// The form of size class LG in this layout: one CTA per instance, or a two-CTA cluster
// (n = 4096 and 8192 by choice, for the solve and the right-hand side separately;
// n = 16384 always).  The solve's u_x hand-off is stored in natural point order by either
// form, so the two kernels may take different forms.
struct PcgKernels {
  template <int LG, int CL>
  static cudaError_t go(const PcgArgs& a, int first, int num, cudaStream_t s) {
    return pcg1d_launch<LG, CL>(a, first, num, s);
  }
  static int ctas(const Layout1d& lay, int l) { return lay.ctas(l); }
};
struct RhsKernels {
  template <int LG, int CL>
  static cudaError_t go(const RhsArgs& a, int first, int num, cudaStream_t s) {
    return rhs1d_launch<LG, CL>(a, first, num, s);
  }
  static int ctas(const Layout1d& lay, int l) { return lay.rhs_ctas(l); }
};

template <int LG, typename K, typename Args>
cudaError_t launch_form(const Layout1d& lay, const Args& a, int first, int num, cudaStream_t s,
                        K) {
  if constexpr (LG > kSmemLog1d) {
    return K::template go<LG, 2>(a, first, num, s);
  } else if constexpr (LG >= kClusterLog1d) {
    return K::ctas(lay, LG) == 2 ? K::template go<LG, 2>(a, first, num, s)
                             : K::template go<LG, 1>(a, first, num, s);
  } else {
    return K::template go<LG, 1>(a, first, num, s);
  }
}

PcgArgs pcg_args(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                 const double* eta, const double* hx, const double* b, double* x,
                 const SolveRec* given, int kind, double rtol, double rtol_inner, int maxit,
                 int max_refine, SolveRec* rec, void* ws, float* coef_df) {
  PcgArgs a;
  a.insts = lay.d_inst;
  a.ids = lay.d_ids;
  a.tw64 = static_cast<const cplx<double>*>(tw64);
  a.twdf = reinterpret_cast<const cplx<df>*>(static_cast<const char*>(tw32) + kTw32Bytes);
  a.eta = eta;
  a.hx = hx;
  a.b = b;
  a.x = x;
  a.given = given;
  a.kind = kind;
  a.rtol = rtol;
  a.rtol_inner = rtol_inner;
  a.maxit = maxit;
  a.max_refine = max_refine;
  a.rec = rec;
  a.ws = static_cast<cplx<double>*>(ws);
  a.coef_df = precision == SGN_PREC_MIXED ? coef_df : nullptr;
  a.precision = precision;
  a.ux = nullptr;
  return a;
}

RhsArgs rhs_args(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                 double g, const double* eta, const double* u, const double* h,
                 const double* hx, double* f_eta, double* f_U, double* scratch) {
  RhsArgs a;
  a.insts = lay.d_inst;
  a.ids = lay.d_ids;
  a.tw64 = static_cast<const cplx<double>*>(tw64);
  a.twdf = reinterpret_cast<const cplx<df>*>(static_cast<const char*>(tw32) + kTw32Bytes);
  a.g = g;
  a.eta = eta;
  a.u = u;
  a.h = h;
  a.hx = hx;
  a.f_eta = f_eta;
  a.f_U = f_U;
  a.scratch = scratch;
  a.P = lay.points;
  a.precision = precision;
  a.ux_given = 0;
  return a;
}

}  // namespace

cudaError_t launch_pcg1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         const double* eta, const double* hx, const double* b, double* x,
                         const SolveRec* given, int kind, double rtol, double rtol_inner,
                         int maxit, int max_refine, SolveRec* rec, void* ws, float* coef_df,
                         cudaStream_t s) {
  const PcgArgs a = pcg_args(lay, tw64, tw32, precision, eta, hx, b, x, given, kind, rtol,
                             rtol_inner, maxit, max_refine, rec, ws, coef_df);
  return d1::for_each_size(lay, s, [&](auto Lc, int first, int num, cudaStream_t cs) {
    return launch_form<decltype(Lc)::value>(lay, a, first, num, cs, PcgKernels{});
  }, [&](int first, int num, cudaStream_t cs) {
    return mr_launch_pcg(lay, first, num, precision, eta, hx, b, x, given, kind, rtol,
                         rtol_inner, maxit, max_refine, rec, ws, cs);
  });
}

cudaError_t launch_pcg1d_ux(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, const double* eta, const double* hx, const double* b,
                            double* x, int kind, double rtol, double rtol_inner, int maxit,
                            int max_refine, SolveRec* rec, void* ws, float* coef_df,
                            double* scratch, cudaStream_t s) {
  PcgArgs a = pcg_args(lay, tw64, tw32, precision, eta, hx, b, x, nullptr, kind, rtol,
                       rtol_inner, maxit, max_refine, rec, ws, coef_df);
  a.ux = scratch;
  // the generic kernels take no u_x hand-off: their right-hand side derives u itself
  return d1::for_each_size(lay, s, [&](auto Lc, int first, int num, cudaStream_t cs) {
    return launch_form<decltype(Lc)::value>(lay, a, first, num, cs, PcgKernels{});
  }, [&](int first, int num, cudaStream_t cs) {
    return mr_launch_pcg(lay, first, num, precision, eta, hx, b, x, nullptr, kind, rtol,
                         rtol_inner, maxit, max_refine, rec, ws, cs);
  });
}

cudaError_t launch_rhs1d(const Layout1d& lay, const void* tw64, const void* tw32, int precision,
                         double g, const double* eta, const double* u, const double* h,
                         const double* hx, double* f_eta, double* f_U, double* scratch,
                         cudaStream_t s) {
  const RhsArgs a = rhs_args(lay, tw64, tw32, precision, g, eta, u, h, hx, f_eta, f_U, scratch);
  return d1::for_each_size(lay, s, [&](auto Lc, int first, int num, cudaStream_t cs) {
    return launch_form<decltype(Lc)::value>(lay, a, first, num, cs, RhsKernels{});
  }, [&](int first, int num, cudaStream_t cs) {
    return mr_launch_rhs(lay, first, num, precision, g, eta, u, h, hx, f_eta, f_U, scratch, cs);
  });
}

cudaError_t launch_rhs1d_ux(const Layout1d& lay, const void* tw64, const void* tw32,
                            int precision, double g, const double* eta, const double* u,
                            const double* h, const double* hx, double* f_eta, double* f_U,
                            double* scratch, cudaStream_t s) {
  RhsArgs a = rhs_args(lay, tw64, tw32, precision, g, eta, u, h, hx, f_eta, f_U, scratch);
  a.ux_given = 1;
  return d1::for_each_size(lay, s, [&](auto Lc, int first, int num, cudaStream_t cs) {
    return launch_form<decltype(Lc)::value>(lay, a, first, num, cs, RhsKernels{});
  }, [&](int first, int num, cudaStream_t cs) {
    return mr_launch_rhs(lay, first, num, precision, g, eta, u, h, hx, f_eta, f_U, scratch, cs);
  });
}

}  // namespace sgn
