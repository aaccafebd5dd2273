"""The PCG robustness suite of §6.2-§6.3 on the GPU, against the oracle.

- Eq:Testproblem with the depth contrast eta0 and the bottom slope h0 swept: the float64
  solve takes the oracle's iteration count, at n = 1024 and at n = 16384 (the two-CTA size),
  and the mixed solve reaches the oracle's solution.  Both run the same Krylov recurrence in
  float64 with different summation orders, so over hundreds of iterations the counts may
  drift apart by rounding: they must agree within max(1, 2%).
- The square-wave depth of the coefficient comparison: optimal against replacement
  coefficients (Remark replacementcoeff), iteration counts equal to the oracle's.
- The 2d elliptical bump (Eq:ellipticalbump) at aspect ratios (1, 1), (1, 20), (1, 40):
  iteration counts equal to the oracle's and growing with the aspect ratio.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SWEEP = [(0.5, 1.0), (1.0, 1.0), (4.0, 1.0), (16.0, 1.0), (1.0, 0.5), (1.0, 2.0), (1.0, 4.0)]


def same_count(got, ref):
    return abs(got - ref) <= max(1, ref // 50)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def S():
    from paper_2506_16045_gb300 import sgn
    ctx = sgn.Context(0)
    yield sgn, ctx
    ctx.close()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n", [1024, 16384])
def test_testproblem_sweep_iterations_match_oracle(S, n):
    sgn, ctx = S
    grid = O.make_grid(1, n, 1.0, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    counts = []
    for eta0, hvar in SWEEP:
        _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
        hx = O.deriv(h, 1.0)
        ref, it_ref, _, c = O.solve_G(eta, hx, b, grid, rtol=1e-12, maxit=5000)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-12, maxit=5000)[0]
        assert info["status"] == 0 and same_count(info["iters"], it_ref), \
            (eta0, hvar, info, it_ref)
        # the two solutions are both within rtol sqrt(kappa_ub) of u* in the G norm
        assert rel(host(x), ref) < 1e-12 * np.sqrt(c["kappa_ub"]) * 10, (eta0, hvar)
        xm = torch.zeros(n, dtype=torch.float64, device="cuda")
        im = sgn.pcg(lay, dev(eta), dev(hx), dev(b), xm, rtol=1e-10, maxit=20000,
                     prec=sgn.PREC_MIXED)[0]
        assert im["status"] == 0 and im["ratio"] <= 1e-10
        assert rel(host(xm), ref) < 1e-10 * np.sqrt(c["kappa_ub"]) * 10, (eta0, hvar)
        counts.append(info["iters"])
    # more contrast, more iterations (§6.2): eta0 = 0.5, 1, 4, 16 and h0 = 0.5, 1, 2, 4
    assert counts[0] <= counts[1] < counts[2] < counts[3]
    assert counts[4] <= counts[1] <= counts[5] <= counts[6]


def test_square_wave_optimal_vs_replacement_coefficients(S):
    sgn, ctx = S
    n = 512
    grid = O.make_grid(1, n, 1.0, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    got = {}
    for eta0 in (0.25, 5.0):
        _, h, eta, b = I.squarewave_1d(n, eta0)
        hx = O.deriv(h, 1.0)
        for kind, ck in (("opt", sgn.COEF_OPT), ("replacement", sgn.COEF_REPLACEMENT)):
            _, it_ref, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-10, maxit=5000, kind=kind)
            P = sgn.precond_coeffs(lay, dev(eta), dev(hx), kind=ck)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-10, maxit=5000, P=P)[0]
            assert info["status"] == 0 and same_count(info["iters"], it_ref), (eta0, kind)
            got[(eta0, kind)] = info["iters"]
    assert got[(0.25, "opt")] + 10 <= got[(0.25, "replacement")], got
    assert abs(got[(5.0, "opt")] - got[(5.0, "replacement")]) <= 1, got


@pytest.mark.parametrize("n", [64, 128])
def test_elliptical_bump_iterations_match_oracle(S, n):
    sgn, ctx = S
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    its = []
    for a, b in ((1.0, 1.0), (1.0, 20.0), (1.0, 40.0)):
        _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, b)
        gh = O.grad(h, (1.0, 1.0))
        ref, it_ref, _, c = O.solve_G(eta, gh, rhs, grid, rtol=1e-10, maxit=5000)
        x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-10, maxit=5000)[0]
        assert info["status"] == 0 and same_count(info["iters"], it_ref), (a, b, info, it_ref)
        assert rel(host(x), ref.ravel()) < 1e-10 * np.sqrt(c["kappa_ub"]) * 10
        its.append(info["iters"])
    assert its[0] < its[1] < its[2], its
