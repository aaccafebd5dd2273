"""GPU parity of the n = 16384 1d path against the CPU oracle (through the C ABI).

n = 16384 is the largest 1d size of the serving workload (1d requests of n = 2^10..2^14).
The solve and the right-hand side run it on thread-block clusters of two CTAs (each CTA
holds half of the points and the modes of one parity), and the float64 helper kernels keep
its transform buffer in global memory.  Every case here mixes n = 16384 instances with
one-CTA sizes in one layout, so a wrong offset or rank mapping shows up as a mismatch in a
neighbour as well.

Tolerances: as in test_gpu_1d.py (float64 <= 1e-12 for single transform pairs, the solve
against the oracle's rtol 1e-14 solution <= 1e-10, mixed precision <= 1e-6 against float64),
and for multi-step runs a bound taken from the oracle's own sensitivity to last-bit changes
of its initial data (third derivatives at k_max = pi n / L ~ 257 amplify rounding).
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BIG = 16384


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
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pack(arrs):
    return np.concatenate([np.asarray(a, dtype=np.float64) for a in arrs])


def unpack(v, offs):
    return [v[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]


MIXED_SIZES = [(BIG, 200.0), (512, 3.0), (BIG, 100.0), (8192, 200.0)]


def shelf_fields(n, L, seed):
    rng = np.random.default_rng(seed)
    x = I.grid_1d(n, L)
    h = I.shelf_1d(x, L, r=0.5 + 0.2 * rng.random(), xs=0.3 * L, w=max(L / 40, 2 * L / n))
    eta = h + 0.2 * np.exp(-((x - 0.6 * L) / (0.05 * L)) ** 2)
    u = 0.3 * np.sin(2 * np.pi * x / L) + 0.05 * np.cos(6 * np.pi * x / L)
    return h, eta, u


def test_cluster_grad_operator_precond(S):
    """Spectral gradient, G apply, preconditioner coefficients and A^{-1} at n = 16384."""
    sgn, ctx = S
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L in MIXED_SIZES])
    hs, etas, us, hxs = [], [], [], []
    for i, (n, L) in enumerate(MIXED_SIZES):
        h, eta, u = shelf_fields(n, L, i)
        u = u + 0.01 * np.random.default_rng(50 + i).standard_normal(n)
        hs.append(h), etas.append(eta), us.append(u), hxs.append(O.deriv(h, L))
    g = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    sgn.spectral_grad(lay, dev(pack(us)), g)
    for (n, L), gi, ui in zip(MIXED_SIZES, unpack(host(g), lay.offsets), us):
        assert rel(gi, O.deriv(ui, L)) < 1e-12, n
    Gu = torch.zeros_like(g)
    sgn.apply_operator(lay, dev(pack(etas)), dev(pack(hxs)), dev(pack(us)), Gu)
    for (n, L), gi, e, hx, u in zip(MIXED_SIZES, unpack(host(Gu), lay.offsets), etas, hxs, us):
        assert rel(gi, O.apply_G_1d(e, hx, u, L)) < 1e-12, n
    got = sgn.precond_coeffs(lay, dev(pack(etas)), dev(pack(hxs)))
    for gp, e, hx in zip(got, etas, hxs):
        w = O.precond_coeffs(e, hx)
        for key in ("sigma", "alpha", "kappa_ub"):
            assert abs(gp[key] - w[key]) <= 1e-14 * abs(w[key]), key
    z = torch.zeros_like(g)
    sgn.precond_solve(lay, got, dev(pack(us)), z)
    for (n, L), zi, u, p in zip(MIXED_SIZES, unpack(host(z), lay.offsets), us, got):
        ref = O.apply_Ainv(u, p["sigma"], p["alpha"], O.make_grid(1, n, L, 1.0))
        assert rel(zi, ref) < 1e-13, n


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("eta0,hvar", [(1.0, 1.0), (1.0, 4.0)])
def test_cluster_pcg_testproblem(S, prec, eta0, hvar):
    """Eq:Testproblem at n = 16384 with u0 = 0 (§6.2): the two-CTA solve equals the oracle's
    solution, and the float64 solve takes the oracle's iteration count."""
    sgn, ctx = S
    n = BIG
    _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    ref, _, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-14, maxit=5000)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    rtol = 1e-12 if prec == "fp64" else 1e-11      # the double-float floor, as at n = 4096
    info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=rtol, maxit=5000, prec=p)[0]
    assert info["status"] == 0 and info["ratio"] <= rtol
    assert rel(host(x), ref) < (1e-10 if prec == "fp64" else 1e-9)
    if prec == "fp64":
        _, it12, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-12, maxit=5000)
        assert abs(info["iters"] - it12) <= 1
    else:
        assert info["refinements"] >= 1


def test_cluster_pcg_batch_equals_alone_bitwise(S):
    """Two n = 16384 clusters and two one-CTA instances in one launch set give bitwise the
    results of each instance solved alone, and recover the velocity b was made from."""
    sgn, ctx = S
    fields = [shelf_fields(n, L, i) for i, (n, L) in enumerate(MIXED_SIZES)]
    hxs = [O.deriv(h, L) for (h, _, _), (n, L) in zip(fields, MIXED_SIZES)]
    bs = [O.apply_G_1d(e, hx, u, L) for (h, e, u), hx, (n, L) in zip(fields, hxs, MIXED_SIZES)]
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L in MIXED_SIZES])
        x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(pack([f[1] for f in fields])), dev(pack(hxs)), dev(pack(bs)),
                       x, rtol=1e-10, prec=prec)
        xb = unpack(host(x), lay.offsets)
        for i, (n, L) in enumerate(MIXED_SIZES):
            assert info[i]["status"] == 0 and info[i]["ratio"] <= 1e-10
            l1 = sgn.Layout(ctx, [sgn.Grid(1, n, L)])
            x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
            sgn.pcg(l1, dev(fields[i][1]), dev(hxs[i]), dev(bs[i]), x1, rtol=1e-10, prec=prec)
            assert np.array_equal(host(x1), xb[i]), (prec, n)
            assert rel(xb[i], fields[i][2]) < 1e-8


def test_cluster_rhs(S):
    """a7 at n = 16384 against the oracle, with the oracle's own last-bit sensitivity as
    the bound (F holds third derivatives)."""
    sgn, ctx = S
    cases = [(BIG, 200.0, 0), (2048, 200.0, 1), (BIG, 400.0, 2)]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L, g=9.81) for n, L, _ in cases])
    hs, etas, us, hxs = [], [], [], []
    for n, L, seed in cases:
        h, eta, u = shelf_fields(n, L, seed)
        hs.append(h), etas.append(eta), us.append(u), hxs.append(O.deriv(h, L))
    fe = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    fU = torch.zeros_like(fe)
    sgn.rhs(lay, dev(pack(etas)), dev(pack(us)), dev(pack(hs)), dev(pack(hxs)), fe, fU)
    for i, (n, L, _) in enumerate(cases):
        re, rU = O.rhs_1d(etas[i], us[i], hs[i], hxs[i], L, 9.81)
        rng = np.random.default_rng(i)
        jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.size))
        pe, pU = O.rhs_1d(jig(etas[i]), jig(us[i]), hs[i], jig(hxs[i]), L, 9.81)
        tol_e = max(1e-13, 20 * rel(pe, re))
        tol_U = max(1e-13, 20 * rel(pU, rU))
        assert rel(unpack(host(fe), lay.offsets)[i], re) < tol_e, (n, tol_e)
        assert rel(unpack(host(fU), lay.offsets)[i], rU) < tol_U, (n, tol_U)
        assert tol_U < 1e-7


def _run_gpu(sgn, ctx, insts, scheme, nsteps, prec, rtol, order=4):
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    eta = dev(pack([c.eta for c in insts]))
    u = dev(pack([c.u for c in insts]))
    h = dev(pack([c.h for c in insts]))
    U = torch.zeros_like(eta)
    gh = torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    dts = [c.dt for c in insts]
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    if scheme == "rk4":
        st.rk4(dts, nsteps, rtol=rtol, prec=p)
    elif scheme == "ab":
        st.abk(order, dts, nsteps, rtol=rtol, prec=p)
    else:
        st.linimp(dts, nsteps, rtol=rtol, prec=p)
    stats = st.stats()
    out = (unpack(host(eta), lay.offsets), unpack(host(U), lay.offsets),
           unpack(host(u), lay.offsets))
    st.close()
    return out, stats


def _run_oracle(c, scheme, nsteps, rtol, order=4, jiggle=None):
    grid = O.make_grid(1, c.n, c.L, c.g)
    eta, u = c.eta, c.u
    if jiggle is not None:
        rng = np.random.default_rng(jiggle)
        eta = eta * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], eta.size))
        u = u * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], u.size))
    st = O.init_state(eta, u, c.h, grid)
    if scheme == "rk4":
        O.run_rk4(st, c.dt, nsteps, rtol)
    elif scheme == "ab":
        O.run_ab(st, order, c.dt, nsteps, rtol)
    else:
        O.run_sbdf2(st, c.dt, nsteps, rtol)
    return st


def _big_shelf():
    dx = 200.0 / BIG
    return I.shelf_case(n=BIG, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0,
                        dt=0.25 * dx / np.sqrt(9.81 * 1.3))


@pytest.mark.parametrize("scheme,order", [("rk4", 0), ("ab", 4), ("linimp", 0)])
def test_cluster_steppers_fp64_match_oracle(S, scheme, order):
    """RK4, AB4 and SBDF2 at n = 16384 (two-CTA solves and right-hand sides; SBDF2's
    A-solve in the global-buffer kernels) against the oracle."""
    sgn, ctx = S
    c = _big_shelf()
    nsteps = 6
    (eta, U, u), stats = _run_gpu(sgn, ctx, [c], scheme, nsteps, "fp64", 1e-13, order or 4)
    ref = _run_oracle(c, scheme, nsteps, 1e-13, order or 4)
    jig = _run_oracle(c, scheme, nsteps, 1e-13, order or 4, jiggle=1)
    zeta_ref = ref.eta - c.h
    tol_z = max(1e-11, 20 * rel(jig.eta - c.h, zeta_ref))
    tol_u = max(1e-11, 20 * rel(jig.u, ref.u))
    tol_U = max(1e-11, 20 * rel(jig.U, ref.U))
    assert rel(eta[0] - c.h, zeta_ref) < tol_z, tol_z
    assert rel(u[0], ref.u) < tol_u, tol_u
    assert rel(U[0], ref.U) < tol_U, tol_U
    assert max(tol_z, tol_u, tol_U) < 1e-8
    assert stats["status"] == 0


def test_cluster_rk4_mixed_precision_within_1e6(S):
    sgn, ctx = S
    c = _big_shelf()
    (eta, U, u), stats = _run_gpu(sgn, ctx, [c], "rk4", 8, "mixed", 1e-11)
    ref = _run_oracle(c, "rk4", 8, 1e-13)
    assert rel(eta[0], ref.eta) < 1e-6 and rel(u[0], ref.u) < 1e-6
    assert stats["status"] == 0 and stats["refinements"] >= stats["solves"]


def test_cluster_ensemble_batch_equals_alone(S):
    """Batched mixed RK4 (graph-replayed from the second step) over n = 8192 and 16384
    instances equals each instance advanced alone, bitwise."""
    sgn, ctx = S
    ens = I.ensemble_1d(count=4, seed=11, kmin=13, kmax=14)
    assert {c.n for c in ens} == {8192, BIG}
    (eta_b, _, u_b), stats = _run_gpu(sgn, ctx, ens, "rk4", 3, "mixed", 1e-10)
    assert stats["status"] == 0
    for i, c in enumerate(ens):
        (eta_1, _, u_1), _ = _run_gpu(sgn, ctx, [c], "rk4", 3, "mixed", 1e-10)
        assert np.array_equal(eta_b[i], eta_1[0]) and np.array_equal(u_b[i], u_1[0]), c.n
