"""Thin Python binding of the C ABI in include/sgn.h (argument marshalling only).

Every numerical step runs in libsgn.so.  Arrays are CUDA float64 tensors (device
pointers are passed through); streams are the current torch CUDA stream unless given.
If the library is missing or no GPU is present, load() raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libsgn.so")

SGN_OK = 0
STATUS_NAMES = {
    0: "SGN_OK", 1: "SGN_ERR_INVALID_ARG", 2: "SGN_ERR_UNSUPPORTED_SIZE", 3: "SGN_ERR_NOMEM",
    4: "SGN_ERR_CUDA", 5: "SGN_ERR_NOT_CONVERGED", 6: "SGN_ERR_BREAKDOWN",
    7: "SGN_ERR_NONPOSITIVE_DEPTH", 8: "SGN_ERR_PENDING", 9: "SGN_ERR_TIMEOUT",
    10: "SGN_ERR_REJECTED",
}
PREC_FP64, PREC_MIXED = 0, 1
COEF_OPT, COEF_REPLACEMENT = 0, 1


class SgnGrid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("Lx", C.c_double),
                ("Ly", C.c_double), ("g", C.c_double)]


class SgnPrecond(C.Structure):
    _fields_ = [("sigma", C.c_double), ("alpha", C.c_double), ("kappa_ub", C.c_double),
                ("flat", C.c_int)]


class SgnPcgInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("rel_resid_Ainv", C.c_double),
                ("status", C.c_int)]


class SgnOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("maxit", C.c_int), ("prec", C.c_int), ("coef", C.c_int),
                ("rtol_inner", C.c_double), ("max_refine", C.c_int)]


class SgnStateStats(C.Structure):
    _fields_ = [("solves", C.c_longlong), ("iterations", C.c_longlong), ("max_iters", C.c_int),
                ("status", C.c_int), ("t", C.c_double), ("step", C.c_longlong),
                ("flops32", C.c_double), ("flops64", C.c_double),
                ("refinements", C.c_longlong), ("sbdf2_stability_warnings", C.c_longlong)]


class SgnRequest(C.Structure):
    _fields_ = [("kind", C.c_int), ("grid", SgnGrid), ("scheme", C.c_int), ("dt", C.c_double),
                ("nsteps", C.c_int), ("opts", SgnOpts), ("eta", C.c_void_p),
                ("u_or_b", C.c_void_p), ("h", C.c_void_p), ("host_memory", C.c_int)]


class SgnResult(C.Structure):
    _fields_ = [("status", C.c_int), ("eta", C.c_void_p), ("u", C.c_void_p), ("U", C.c_void_p),
                ("info", SgnPcgInfo), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


REQ_SOLVE, REQ_RUN = 0, 1
SCHEME_RK4, SCHEME_AB2, SCHEME_AB3, SCHEME_AB4, SCHEME_LINIMP = 0, 2, 3, 4, 5
SGN_ERR_PENDING = 8

# (name, restype, argtypes) of every exported entry point declared in include/sgn.h
_VP = C.c_void_p
_DP = C.c_void_p       # device pointers travel as integers
SIGNATURES = [
    ("sgn_create", C.c_int, [C.POINTER(_VP), C.c_int, C.c_size_t]),
    ("sgn_destroy", None, [_VP]),
    ("sgn_last_error", C.c_char_p, [_VP]),
    ("sgn_status_string", C.c_char_p, [C.c_int]),
    ("sgn_layout_create", C.c_int, [_VP, C.c_int, C.POINTER(SgnGrid), C.POINTER(_VP)]),
    ("sgn_layout_destroy", None, [_VP]),
    ("sgn_layout_points", C.c_longlong, [_VP]),
    ("sgn_layout_offsets", C.c_int, [_VP, C.POINTER(C.c_longlong)]),
    ("sgn_layout_set_form", C.c_int, [_VP, C.c_int, C.c_int]),
    ("sgn_layout_get_form", C.c_int, [_VP, C.c_int, C.POINTER(C.c_int)]),
    ("sgn_layout_set_forms", C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
    ("sgn_layout_get_forms", C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("sgn_layout_set_form2d", C.c_int, [_VP, C.c_int, C.c_int]),
    ("sgn_layout_get_form2d", C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("sgn_layout_set_radix2d", C.c_int, [_VP, C.c_int]),
    ("sgn_layout_get_radix2d", C.c_int, [_VP, C.POINTER(C.c_int)]),
    ("sgn_layout_set_unit_threads2d", C.c_int, [_VP, C.c_int]),
    ("sgn_layout_get_unit_threads2d", C.c_int, [_VP, C.POINTER(C.c_int)]),
    ("sgn_spectral_grad", C.c_int, [_VP, _VP, _DP, _DP, _VP]),
    ("sgn_precond_coeffs", C.c_int, [_VP, _VP, _DP, _DP, C.c_int, C.POINTER(SgnPrecond), _VP]),
    ("sgn_apply_operator", C.c_int, [_VP, _VP, _DP, _DP, _DP, _DP, _VP]),
    ("sgn_precond_solve", C.c_int, [_VP, _VP, C.POINTER(SgnPrecond), _DP, _DP, _VP]),
    ("sgn_pcg", C.c_int, [_VP, _VP, _DP, _DP, C.POINTER(SgnPrecond), _DP, _DP, C.c_double,
                          C.c_int, C.c_int, C.POINTER(SgnPcgInfo), _VP]),
    ("sgn_pcg_async", C.c_int, [_VP, _VP, _DP, _DP, _DP, _DP, C.c_double, C.c_int, C.c_int,
                                _VP, _VP]),
    ("sgn_gmres", C.c_int, [_VP, _VP, _DP, _DP, C.POINTER(SgnPrecond), _DP, _DP, C.c_double,
                            C.c_int, C.c_int, C.POINTER(SgnPcgInfo), _VP]),
    ("sgn_rhs", C.c_int, [_VP, _VP, _DP, _DP, _DP, _DP, _DP, _DP, _VP]),
    ("sgn_state_create", C.c_int, [_VP, _VP, _DP, _DP, _DP, _DP, _DP, C.POINTER(_VP)]),
    ("sgn_state_init", C.c_int, [_VP, _VP]),
    ("sgn_step_rk4", C.c_int, [_VP, C.POINTER(C.c_double), C.c_int, C.POINTER(SgnOpts), _VP]),
    ("sgn_step_rk4_nc", C.c_int, [_VP, C.POINTER(C.c_double), C.c_int, C.POINTER(SgnOpts),
                                  _VP]),
    ("sgn_step_abk", C.c_int, [_VP, C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(SgnOpts),
                               _VP]),
    ("sgn_step_linimp", C.c_int, [_VP, C.POINTER(C.c_double), C.c_int, C.POINTER(SgnOpts), _VP]),
    ("sgn_state_set_dealias", C.c_int, [_VP, C.c_int]),
    ("sgn_state_set_forcing", C.c_int, [_VP, C.c_int, _DP, _DP, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    ("sgn_state_autotune", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(SgnOpts), _VP,
                                     C.POINTER(C.c_double)]),
    ("sgn_state_get_stats", C.c_int, [_VP, C.POINTER(SgnStateStats)]),
    ("sgn_state_free", None, [_VP]),
    ("sgn_pcg1d_noalloc", C.c_int, [C.c_int, C.c_double, _DP, _DP, _DP, _DP, C.c_double, C.c_int,
                                    C.c_int, C.POINTER(SgnPcgInfo), _VP]),
    ("sgn_server_create", C.c_int, [_VP, C.c_double, C.POINTER(_VP)]),
    ("sgn_batch_submit", C.c_int, [_VP, C.POINTER(SgnRequest), C.POINTER(C.c_uint64)]),
    ("sgn_batch_poll", C.c_int, [_VP, C.c_uint64, C.POINTER(SgnResult)]),
    ("sgn_result_release", C.c_int, [_VP, C.c_uint64]),
    ("sgn_server_destroy", None, [_VP]),
    ("sgn_clock", C.c_double, []),
    ("sgn_profile_enable", C.c_int, [_VP, C.c_int]),
    ("sgn_profile_read", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    ("sgn_profile_inner2d", C.c_int, [_VP, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
]

_lib = None


def load(path: str = LIBPATH):
    """Load libsgn.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsgn.so not found at {path}: build it with "
                           "`python -m paper_2506_16045_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SgnError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


def _ptr(t):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


def _vptr(t):
    """Device address of a contiguous CUDA tensor of any dtype (raw byte buffers)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclass
class Grid:
    dim: int
    nx: int
    Lx: float
    g: float = 9.81
    ny: int = 1
    Ly: float = 1.0

    def c(self):
        return SgnGrid(self.dim, self.nx, self.ny, self.Lx, self.Ly, self.g)

    @property
    def points(self):
        return self.nx * self.ny


class Context:
    """Owns an sgn_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        s = self.lib.sgn_create(C.byref(h), device, 0)
        if s != SGN_OK:
            raise SgnError(s, "sgn_create")
        self.h = h
        self.device = device
        self._children = []            # weak references to layouts, states and servers

    def _adopt(self, obj):
        self._children.append(weakref.ref(obj))

    def check(self, s, what=""):
        if s != SGN_OK:
            msg = self.lib.sgn_last_error(self.h)
            raise SgnError(s, f"{what}: {msg.decode() if msg else ''}")

    def profile(self, on: bool):
        self.check(self.lib.sgn_profile_enable(self.h, 1 if on else 0), "sgn_profile_enable")

    def profile_read(self):
        """Synchronises the profiled launch groups; returns dict of summed ms and counts."""
        pm, pc, rm, rc = C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong()
        self.check(self.lib.sgn_profile_read(self.h, C.byref(pm), C.byref(pc), C.byref(rm),
                                             C.byref(rc)), "sgn_profile_read")
        return dict(pcg_ms=pm.value, pcg_calls=pc.value, rhs_ms=rm.value, rhs_calls=rc.value)

    def close(self):
        """Frees the context after everything created from it (newest first)."""
        if self.h:
            for ref in reversed(self._children):
                obj = ref()
                if obj is not None:
                    obj.close()
            self._children = []
            self.lib.sgn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Layout:
    """A packed batch of instances (sgn_layout)."""

    def __init__(self, ctx: Context, grids: Sequence[Grid]):
        self.ctx = ctx
        self.grids = list(grids)
        arr = (SgnGrid * len(self.grids))(*[g.c() for g in self.grids])
        h = C.c_void_p()
        ctx.check(ctx.lib.sgn_layout_create(ctx.h, len(self.grids), arr, C.byref(h)),
                  "sgn_layout_create")
        self.h = h
        self.count = len(self.grids)
        self.points = ctx.lib.sgn_layout_points(h)
        offs = (C.c_longlong * (self.count + 1))()
        ctx.check(ctx.lib.sgn_layout_offsets(h, offs), "sgn_layout_offsets")
        self.offsets = list(offs)
        self.dim = self.grids[0].dim
        ctx._adopt(self)

    def set_form(self, log2n, ctas):
        """One CTA (1) or a two-CTA cluster (2) per instance for the class n = 2^log2n."""
        self.ctx.check(self.ctx.lib.sgn_layout_set_form(self.h, log2n, ctas),
                       "sgn_layout_set_form")

    def form(self, log2n):
        c = C.c_int()
        self.ctx.check(self.ctx.lib.sgn_layout_get_form(self.h, log2n, C.byref(c)),
                       "sgn_layout_get_form")
        return c.value

    def set_forms(self, log2n, solve_ctas, rhs_ctas):
        """Separate forms for the class's solve and right-hand side."""
        self.ctx.check(self.ctx.lib.sgn_layout_set_forms(self.h, log2n, solve_ctas, rhs_ctas),
                       "sgn_layout_set_forms")

    def forms(self, log2n):
        """(solve CTAs, right-hand-side CTAs) per instance of the class n = 2^log2n."""
        a, b = C.c_int(), C.c_int()
        self.ctx.check(self.ctx.lib.sgn_layout_get_forms(self.h, log2n, C.byref(a), C.byref(b)),
                       "sgn_layout_get_forms")
        return a.value, b.value

    def set_form2d(self, inner, tile_width=0):
        """sgn_layout_set_form2d: inner 0 = persistent inner solve, 1 = four kernels per
        inner iteration; tile_width 0 = automatic (one column per tile), or 1."""
        self.ctx.check(self.ctx.lib.sgn_layout_set_form2d(self.h, inner, tile_width),
                       "sgn_layout_set_form2d")

    def profile_inner2d(self, on):
        """sgn_profile_inner2d: (ms, launches, inner iterations) recorded since the last
        call; then recording on or off."""
        ms, n, it = C.c_double(), C.c_longlong(), C.c_longlong()
        self.ctx.check(self.ctx.lib.sgn_profile_inner2d(self.h, 1 if on else 0, C.byref(ms),
                                                        C.byref(n), C.byref(it)),
                       "sgn_profile_inner2d")
        return ms.value, n.value, it.value

    def set_radix2d(self, max_radix):
        """sgn_layout_set_radix2d: the persistent inner solve's transform stages up to radix
        8 (default, also 0) or 16."""
        self.ctx.check(self.ctx.lib.sgn_layout_set_radix2d(self.h, max_radix),
                       "sgn_layout_set_radix2d")

    def set_unit_threads2d(self, threads):
        """sgn_layout_set_unit_threads2d: threads per unit of the persistent 2d inner solve
        (128, 256, or 0: chosen by the unit count)."""
        self.ctx.check(self.ctx.lib.sgn_layout_set_unit_threads2d(self.h, threads),
                       "sgn_layout_set_unit_threads2d")

    def unit_threads2d(self):
        r = C.c_int()
        self.ctx.check(self.ctx.lib.sgn_layout_get_unit_threads2d(self.h, C.byref(r)),
                       "sgn_layout_get_unit_threads2d")
        return r.value

    def radix2d(self):
        r = C.c_int()
        self.ctx.check(self.ctx.lib.sgn_layout_get_radix2d(self.h, C.byref(r)),
                       "sgn_layout_get_radix2d")
        return r.value

    def form2d(self):
        i, t = C.c_int(), C.c_int()
        self.ctx.check(self.ctx.lib.sgn_layout_get_form2d(self.h, C.byref(i), C.byref(t)),
                       "sgn_layout_get_form2d")
        return i.value, t.value

    def close(self):
        if self.h:
            self.ctx.lib.sgn_layout_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spectral_grad(lay: Layout, f, gradf, stream=None):
    lay.ctx.check(lay.ctx.lib.sgn_spectral_grad(lay.ctx.h, lay.h, _ptr(f), _ptr(gradf),
                                                _stream(stream)), "sgn_spectral_grad")


def precond_coeffs(lay: Layout, eta, gradh, kind=COEF_OPT, stream=None):
    out = (SgnPrecond * lay.count)()
    lay.ctx.check(lay.ctx.lib.sgn_precond_coeffs(lay.ctx.h, lay.h, _ptr(eta), _ptr(gradh), kind,
                                                 out, _stream(stream)), "sgn_precond_coeffs")
    return [dict(sigma=p.sigma, alpha=p.alpha, kappa_ub=p.kappa_ub, flat=bool(p.flat)) for p in out]


def apply_operator(lay: Layout, eta, gradh, u, Gu, stream=None):
    lay.ctx.check(lay.ctx.lib.sgn_apply_operator(lay.ctx.h, lay.h, _ptr(eta), _ptr(gradh), _ptr(u),
                                                 _ptr(Gu), _stream(stream)), "sgn_apply_operator")


def _precond_array(lay, P):
    arr = (SgnPrecond * lay.count)()
    for i, p in enumerate(P):
        arr[i] = SgnPrecond(p["sigma"], p["alpha"], p.get("kappa_ub", 0.0), int(p.get("flat", 0)))
    return arr


def precond_solve(lay: Layout, P, r, z, stream=None):
    lay.ctx.check(lay.ctx.lib.sgn_precond_solve(lay.ctx.h, lay.h, _precond_array(lay, P), _ptr(r),
                                                _ptr(z), _stream(stream)), "sgn_precond_solve")


def pcg(lay: Layout, eta, gradh, b, x, rtol=1e-12, maxit=1000, prec=PREC_FP64, P=None,
        info=True, stream=None, check=True):
    """Solve G x = b (x holds the initial guess).  Returns per-instance info dicts (or None)."""
    inf = (SgnPcgInfo * lay.count)() if info else None
    parr = _precond_array(lay, P) if P is not None else None
    s = lay.ctx.lib.sgn_pcg(lay.ctx.h, lay.h, _ptr(eta), _ptr(gradh), parr, _ptr(b), _ptr(x), rtol,
                            maxit, prec, inf, _stream(stream))
    if check:
        lay.ctx.check(s, "sgn_pcg")
    if not info:
        return None
    return [dict(iters=i.iters, refinements=i.refinements, ratio=i.rel_resid_Ainv,
                 status=i.status) for i in inf]


PCG_INFO_BYTES = C.sizeof(SgnPcgInfo)


def pcg_async(lay: Layout, eta, gradh, b, x, info_dev, rtol=1e-12, maxit=1000, prec=PREC_FP64,
              stream=None):
    """sgn_pcg_async: the solve with optimal coefficients and its report written to device
    memory `info_dev` (count * PCG_INFO_BYTES bytes, e.g. a uint8 CUDA tensor); nothing
    synchronises.  Decode the bytes with pcg_info_from_bytes once the stream has finished."""
    lay.ctx.check(lay.ctx.lib.sgn_pcg_async(lay.ctx.h, lay.h, _ptr(eta), _ptr(gradh), _ptr(b),
                                            _ptr(x), rtol, maxit, prec, _vptr(info_dev),
                                            _stream(stream)), "sgn_pcg_async")


def pcg_info_from_bytes(raw: bytes, count: int):
    """The per-instance sgn_pcg_info records in `raw` (host bytes) as dicts."""
    arr = (SgnPcgInfo * count).from_buffer_copy(raw[:count * PCG_INFO_BYTES])
    return [dict(iters=i.iters, refinements=i.refinements, ratio=i.rel_resid_Ainv,
                 status=i.status) for i in arr]


def gmres(lay: Layout, eta, gradh, b, x, rtol=1e-10, restart=30, maxit=1000, P=None,
          info=True, stream=None, check=True):
    """sgn_gmres: restarted GMRES right-preconditioned by A, in the A^{-1} inner product (x
    holds the initial guess).  Returns per-instance info dicts: iters = Arnoldi steps,
    cycles, ratio = the final sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b), status."""
    inf = (SgnPcgInfo * lay.count)() if info else None
    parr = _precond_array(lay, P) if P is not None else None
    s = lay.ctx.lib.sgn_gmres(lay.ctx.h, lay.h, _ptr(eta), _ptr(gradh), parr, _ptr(b), _ptr(x),
                              rtol, restart, maxit, inf, _stream(stream))
    if check:
        lay.ctx.check(s, "sgn_gmres")
    if not info:
        return None
    return [dict(iters=i.iters, cycles=i.refinements, ratio=i.rel_resid_Ainv, status=i.status)
            for i in inf]


def pcg1d_noalloc(n, L, eta, gradh, b, x, rtol=1e-12, maxit=1000, prec=PREC_FP64, stream=None):
    """sgn_pcg1d_noalloc: the single-instance 1d solve without any device allocation (for
    callers that cannot allocate once running).  Returns (status, info dict)."""
    lib = load()
    inf = SgnPcgInfo()
    s = lib.sgn_pcg1d_noalloc(n, L, _ptr(eta), _ptr(gradh), _ptr(b), _ptr(x), rtol, maxit, prec,
                              C.byref(inf), _stream(stream))
    return s, dict(iters=inf.iters, refinements=inf.refinements, ratio=inf.rel_resid_Ainv,
                   status=inf.status)


def rhs(lay: Layout, eta, u, h, gradh, f_eta, f_U, stream=None):
    lay.ctx.check(lay.ctx.lib.sgn_rhs(lay.ctx.h, lay.h, _ptr(eta), _ptr(u), _ptr(h), _ptr(gradh),
                                      _ptr(f_eta), _ptr(f_U), _stream(stream)), "sgn_rhs")


class State:
    """sgn_state bound to caller-owned tensors eta, U, u, h, gradh (packed)."""

    def __init__(self, lay: Layout, eta, U, u, h, gradh):
        self.lay = lay
        self.tensors = (eta, U, u, h, gradh)
        hh = C.c_void_p()
        lay.ctx.check(lay.ctx.lib.sgn_state_create(lay.ctx.h, lay.h, _ptr(eta), _ptr(U), _ptr(u),
                                                   _ptr(h), _ptr(gradh), C.byref(hh)),
                      "sgn_state_create")
        self.h = hh
        lay.ctx._adopt(self)

    def init(self, stream=None):
        self.lay.ctx.check(self.lay.ctx.lib.sgn_state_init(self.h, _stream(stream)),
                           "sgn_state_init")

    @staticmethod
    def _opts(rtol, maxit, prec, coef, rtol_inner, max_refine):
        return SgnOpts(rtol, maxit, prec, coef, rtol_inner, max_refine)

    def _dt(self, dt):
        n = self.lay.count
        vals = [float(dt)] * n if not hasattr(dt, "__len__") else [float(v) for v in dt]
        return (C.c_double * n)(*vals)

    def rk4(self, dt, nsteps, rtol=1e-12, maxit=2000, prec=PREC_FP64, coef=COEF_OPT,
            rtol_inner=0.0, max_refine=0, stream=None):
        o = self._opts(rtol, maxit, prec, coef, rtol_inner, max_refine)
        self.lay.ctx.check(self.lay.ctx.lib.sgn_step_rk4(self.h, self._dt(dt), nsteps, C.byref(o),
                                                         _stream(stream)), "sgn_step_rk4")

    def rk4_nc(self, dt, nsteps, rtol=1e-12, maxit=2000, prec=PREC_FP64, coef=COEF_OPT,
               rtol_inner=0.0, max_refine=0, stream=None):
        """sgn_step_rk4_nc: RK4 on the non-constraint form (eta, u), 1d and 2d."""
        o = self._opts(rtol, maxit, prec, coef, rtol_inner, max_refine)
        self.lay.ctx.check(self.lay.ctx.lib.sgn_step_rk4_nc(self.h, self._dt(dt), nsteps,
                                                            C.byref(o), _stream(stream)),
                           "sgn_step_rk4_nc")

    def abk(self, order, dt, nsteps, rtol=1e-12, maxit=2000, prec=PREC_FP64, coef=COEF_OPT,
            rtol_inner=0.0, max_refine=0, stream=None):
        o = self._opts(rtol, maxit, prec, coef, rtol_inner, max_refine)
        self.lay.ctx.check(self.lay.ctx.lib.sgn_step_abk(self.h, order, self._dt(dt), nsteps,
                                                         C.byref(o), _stream(stream)),
                           "sgn_step_abk")

    def linimp(self, dt, nsteps, rtol=1e-12, maxit=2000, prec=PREC_FP64, coef=COEF_OPT,
               rtol_inner=0.0, max_refine=0, stream=None):
        o = self._opts(rtol, maxit, prec, coef, rtol_inner, max_refine)
        self.lay.ctx.check(self.lay.ctx.lib.sgn_step_linimp(self.h, self._dt(dt), nsteps,
                                                            C.byref(o), _stream(stream)),
                           "sgn_step_linimp")

    def autotune(self, dt, rtol=1e-12, maxit=2000, prec=PREC_FP64, coef=COEF_OPT,
                 rtol_inner=0.0, max_refine=0, stream=None):
        """Times the layout's kernel forms on RK4 steps of this state's problem and keeps the
        fastest (the state is restored); returns the winning time per step (ms)."""
        o = self._opts(rtol, maxit, prec, coef, rtol_inner, max_refine)
        ms = C.c_double()
        self.lay.ctx.check(self.lay.ctx.lib.sgn_state_autotune(self.h, self._dt(dt), C.byref(o),
                                                               _stream(stream), C.byref(ms)),
                           "sgn_state_autotune")
        return ms.value

    def set_dealias(self, on=True):
        """2/3-rule dealiasing of every new time level (sgn_state_set_dealias)."""
        self.lay.ctx.check(self.lay.ctx.lib.sgn_state_set_dealias(self.h, 1 if on else 0),
                           "sgn_state_set_dealias")

    def set_forcing(self, phi_eta, phi_U, omega, theta):
        """External forcing sum_k cos(omega_k t + theta_k) (phi_eta_k, phi_U_k) (device
        tensors [K][P] and [K][d P]); K = 0 (empty omega) removes it.  The tensors are kept
        referenced here, since the library reads them at every step."""
        K = len(omega)
        om = (C.c_double * max(K, 1))(*[float(v) for v in omega])
        th = (C.c_double * max(K, 1))(*[float(v) for v in theta])
        self._forcing = (phi_eta, phi_U) if K else None
        self.lay.ctx.check(self.lay.ctx.lib.sgn_state_set_forcing(
            self.h, K, _ptr(phi_eta) if K else None, _ptr(phi_U) if K else None, om, th),
            "sgn_state_set_forcing")

    def stats(self):
        st = SgnStateStats()
        self.lay.ctx.check(self.lay.ctx.lib.sgn_state_get_stats(self.h, C.byref(st)),
                           "sgn_state_get_stats")
        return dict(solves=st.solves, iterations=st.iterations, max_iters=st.max_iters,
                    status=st.status, t=st.t, step=st.step, flops32=st.flops32,
                    flops64=st.flops64, refinements=st.refinements,
                    sbdf2_stability_warnings=st.sbdf2_stability_warnings)

    def close(self):
        if self.h:
            self.lay.ctx.lib.sgn_state_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (sgn_server) on the context's device."""

    def __init__(self, ctx: Context, budget_fraction: float = 0.0):
        self.ctx = ctx
        self.lib = ctx.lib
        h = C.c_void_p()
        ctx.check(self.lib.sgn_server_create(ctx.h, budget_fraction, C.byref(h)),
                  "sgn_server_create")
        self.h = h
        ctx._adopt(self)

    def submit(self, kind, grid: Grid, eta, u_or_b, h, scheme=SCHEME_RK4, dt=0.0, nsteps=0,
               rtol=1e-10, maxit=4000, prec=PREC_MIXED, coef=COEF_OPT, host=False):
        """Queue a request; arrays are CUDA float64 tensors (host=False) or contiguous numpy
        float64 arrays (host=True).  Returns (status, ticket)."""
        if host:
            import numpy as np
            keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (eta, u_or_b, h)]
            ptrs = [a.ctypes.data for a in keep]
        else:
            ptrs = [_ptr(eta), _ptr(u_or_b), _ptr(h)]
        req = SgnRequest(kind, grid.c(), scheme, dt, nsteps,
                         SgnOpts(rtol, maxit, prec, coef, 0.0, 0), ptrs[0], ptrs[1], ptrs[2],
                         1 if host else 0)
        t = C.c_uint64()
        s = self.lib.sgn_batch_submit(self.h, C.byref(req), C.byref(t))
        return s, t.value

    def poll(self, ticket):
        """None while pending, else a dict with status, device pointers, info and times."""
        r = SgnResult()
        s = self.lib.sgn_batch_poll(self.h, ticket, C.byref(r))
        if s == SGN_ERR_PENDING:
            return None
        return dict(status=r.status, eta=r.eta, u=r.u, U=r.U, iters=r.info.iters,
                    refinements=r.info.refinements, ratio=r.info.rel_resid_Ainv,
                    t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done)

    def release(self, ticket):
        return self.lib.sgn_result_release(self.h, ticket)

    def close(self):
        if self.h:
            self.lib.sgn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CudaArray:
    """Minimal __cuda_array_interface__ wrapper of a device float64 array (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3}


def device_array(ptr, n):
    """A CUDA float64 tensor copy of the n values at device address ptr (e.g. a result)."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, n), device="cuda").clone()
