"""The allocation-free solve (sgn_pcg1d_noalloc) gives the same answer as sgn_pcg and the
oracle, and allocates no device memory after its first call.

The entry point serves callers that cannot allocate device memory once running (a fixed
memory pool, a frozen-heap host, a callback inside another code's time loop).  Its scratch
is static device memory shared by every call, so this file checks two calls in a row (the
second sees the first call's leftovers) against the regular entry point, with the
tolerance the other PCG parity tests use, and both against the oracle's solve.  The first
call on a device may load the library's module (lazy loading places the static arrays
then), so the free-memory check starts after a warm-up call.  It is named to be collected
last.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_sgn_pcg_on_two_calls_in_a_row():
    from paper_2506_16045_gb300 import sgn
    ctx = sgn.Context(0)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    cases = [(4096, 4.0, 1.0, sgn.PREC_MIXED), (1024, 1.0, 1.0, sgn.PREC_FP64),
             (4096, 1.0, 4.0, sgn.PREC_MIXED)]
    for n, eta0, hvar, prec in cases:
        _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
        hx = O.deriv(h, 1.0)
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
        x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        # mixed precision: 1e-11 (its double-float residual floor is near 1e-12 on h0 = 4)
        rtol = 1e-12 if prec == sgn.PREC_FP64 else 1e-11
        info_ref = sgn.pcg(lay, d(eta), d(hx), d(b), x_ref, rtol=rtol, maxit=5000, prec=prec)[0]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = sgn.pcg1d_noalloc(n, 1.0, d(eta), d(hx), d(b), x, rtol=rtol, maxit=5000,
                                     prec=prec)
        torch.cuda.synchronize()
        assert st == sgn.SGN_OK and info["status"] == sgn.SGN_OK
        assert info["iters"] == info_ref["iters"]
        assert _rel(x.cpu().numpy(), x_ref.cpu().numpy()) < 1e-10
        # against the oracle's float64 solve of the same system
        x_or = O.solve_G(eta, hx, b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-13)[0]
        assert _rel(x.cpu().numpy(), x_or) < 1e-9
    ctx.close()


def test_noalloc_allocates_nothing_after_its_first_call():
    """After one warm-up call, further calls leave the device's free memory unchanged."""
    from paper_2506_16045_gb300 import sgn
    n = 2048
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    eta_d, hx_d, b_d = d(eta), d(hx), d(b)
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    st, _ = sgn.pcg1d_noalloc(n, 1.0, eta_d, hx_d, b_d, xs[0], rtol=1e-11, maxit=2000,
                              prec=sgn.PREC_MIXED)
    assert st == sgn.SGN_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for x in xs[1:]:
        st, _ = sgn.pcg1d_noalloc(n, 1.0, eta_d, hx_d, b_d, x, rtol=1e-11, maxit=2000,
                                  prec=sgn.PREC_MIXED)
        assert st == sgn.SGN_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = O.solve_G(eta, hx, b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-13)[0]
    for x in xs:
        assert _rel(x.cpu().numpy(), ref) < 1e-9


def test_noalloc_rejects_sizes_beyond_its_maximum():
    from paper_2506_16045_gb300 import sgn
    big = 2 * 8192
    z = torch.zeros(big, dtype=torch.float64, device="cuda")
    st, _ = sgn.pcg1d_noalloc(big, 1.0, z, z, z, z)
    assert st == 2                      # SGN_ERR_UNSUPPORTED_SIZE
    st, _ = sgn.pcg1d_noalloc(96, 1.0, z, z, z, z)
    assert st == 2
