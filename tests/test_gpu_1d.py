"""GPU parity of the 1d CUDA path against the CPU oracle (through the C ABI).

Tolerances: float64 paths <= 1e-11 relative L2 (tighter where the operation is a single
transform pair); the mixed float32/float64 path <= 1e-6 relative L2 against float64.
"""
import math

import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


RAGGED = [(8, 1.0), (16, 2.0), (64, 7.5), (256, 100.0), (512, 3.0), (1024, 1.0), (2048, 200.0),
          (4096, 200.0), (8192, 200.0), (128, 0.5)]


def shelf_fields(n, L, seed):
    rng = np.random.default_rng(seed)
    x = I.grid_1d(n, L)
    h = I.shelf_1d(x, L, r=0.5 + 0.2 * rng.random(), xs=0.3 * L, w=max(L / 40, 2 * L / n))
    eta = h + 0.2 * np.exp(-((x - 0.6 * L) / (0.05 * L)) ** 2)
    u = 0.3 * np.sin(2 * np.pi * x / L) + 0.1 * rng.standard_normal(n) * 0 + \
        0.05 * np.cos(6 * np.pi * x / L)
    return h, eta, u


def test_spectral_grad_ragged_batch(S):
    sgn, ctx = S
    grids = [sgn.Grid(1, n, L) for n, L in RAGGED]
    lay = sgn.Layout(ctx, grids)
    fs = [shelf_fields(n, L, i)[0] + np.random.default_rng(i).standard_normal(n) * 0.01
          for i, (n, L) in enumerate(RAGGED)]
    f = dev(pack(fs))
    g = torch.zeros_like(f)
    sgn.spectral_grad(lay, f, g)
    out = unpack(host(g), lay.offsets)
    for (n, L), fi, gi in zip(RAGGED, fs, out):
        assert rel(gi, O.deriv(fi, L)) < 1e-12, n


def test_apply_operator_ragged_batch(S):
    sgn, ctx = S
    grids = [sgn.Grid(1, n, L) for n, L in RAGGED]
    lay = sgn.Layout(ctx, grids)
    hs, etas, us, hxs, refs = [], [], [], [], []
    for i, (n, L) in enumerate(RAGGED):
        h, eta, u = shelf_fields(n, L, i)
        u = u + 0.01 * np.random.default_rng(100 + i).standard_normal(n)
        hx = O.deriv(h, L)
        hs.append(h), etas.append(eta), us.append(u), hxs.append(hx)
        refs.append(O.apply_G_1d(eta, hx, u, L))
    Gu = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    sgn.apply_operator(lay, dev(pack(etas)), dev(pack(hxs)), dev(pack(us)), Gu)
    for (n, L), gi, ri in zip(RAGGED, unpack(host(Gu), lay.offsets), refs):
        assert rel(gi, ri) < 1e-12, n


def test_apply_operator_matches_dense_weak_form(S):
    """Small n: the CUDA G against the oracle's dense W^T M W (Def:MatrixM)."""
    sgn, ctx = S
    n = 32
    _, h, eta, _ = I.testproblem_1d(n, 4.0, 1.0)
    hx = O.deriv(h, 1.0)
    Gd = O.dense_G_1d(eta, hx, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    for seed in range(3):
        u = np.random.default_rng(seed).standard_normal(n)
        Gu = torch.zeros(n, dtype=torch.float64, device="cuda")
        sgn.apply_operator(lay, dev(eta), dev(hx), dev(u), Gu)
        assert rel(host(Gu), Gd @ u) < 1e-13


def test_precond_coeffs_and_solve(S):
    sgn, ctx = S
    cases = [(64, 1.0, 1.0, 1.0), (256, 1.0, 4.0, 0.0), (1024, 1.0, 0.5, 4.0)]
    grids = [sgn.Grid(1, n, L) for n, L, _, _ in cases]
    lay = sgn.Layout(ctx, grids)
    etas, hxs, want = [], [], []
    for n, L, eta0, hv in cases:
        _, h, eta, _ = I.testproblem_1d(n, eta0, hv)
        hx = O.deriv(h, 1.0) if hv else np.zeros(n)
        etas.append(eta), hxs.append(hx)
        want.append(O.precond_coeffs(eta, hx))
    got = sgn.precond_coeffs(lay, dev(pack(etas)), dev(pack(hxs)))
    for g, w in zip(got, want):
        for key in ("sigma", "alpha", "kappa_ub"):
            assert abs(g[key] - w[key]) <= 1e-14 * abs(w[key]), key
        assert g["flat"] == w["flat"]
    gotr = sgn.precond_coeffs(lay, dev(pack(etas)), dev(pack(hxs)), kind=sgn.COEF_REPLACEMENT)
    for g, eta, hx in zip(gotr, etas, hxs):
        w = O.precond_coeffs(eta, hx, "replacement")
        assert abs(g["sigma"] - w["sigma"]) <= 1e-14 * w["sigma"]
    r = [np.random.default_rng(i).standard_normal(n) for i, (n, *_ ) in enumerate(cases)]
    z = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    sgn.precond_solve(lay, got, dev(pack(r)), z)
    for (n, L, _, _), zi, ri, p in zip(cases, unpack(host(z), lay.offsets), r, got):
        ref = O.apply_Ainv(ri, p["sigma"], p["alpha"], O.make_grid(1, n, L, 1.0))
        assert rel(zi, ref) < 1e-13


def test_precond_coeffs_rejects_nonpositive_depth(S):
    sgn, ctx = S
    lay = sgn.Layout(ctx, [sgn.Grid(1, 64, 1.0)])
    eta = np.ones(64)
    eta[10] = -0.1
    with pytest.raises(sgn.SgnError) as e:
        sgn.precond_coeffs(lay, dev(eta), dev(np.zeros(64)))
    assert e.value.status == 7


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,eta0,hvar", [(64, 1.0, 1.0), (256, 1.0, 1.0), (1024, 4.0, 1.0),
                                         (4096, 1.0, 4.0), (8192, 1.0, 1.0)])
def test_pcg_testproblem(S, prec, n, eta0, hvar):
    """Eq:Testproblem with u0 = 0 (§6.2): the CUDA solve equals the oracle's solution."""
    sgn, ctx = S
    _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    ref, it_ref, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-14, maxit=5000)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    # The double-float residual of the mixed path carries ~2^-48 relative rounding, which the
    # operator's range (eta (1 + h_x^2) up to ~5e3 here) lifts to a floor near 1e-12 in the
    # relative A^{-1} residual on the h0 = 4 problems, so the mixed solve is asked for 1e-11.
    rtol = 1e-12 if prec == "fp64" else 1e-11
    info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=rtol, maxit=5000, prec=p)[0]
    assert info["status"] == 0 and info["ratio"] <= rtol
    assert rel(host(x), ref) < (1e-10 if prec == "fp64" else 1e-9)
    if prec == "fp64":
        _, it12, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-12, maxit=5000)
        assert abs(info["iters"] - it12) <= 1
    else:
        assert info["refinements"] >= 1


def test_pcg_batch_equals_alone_bitwise(S):
    sgn, ctx = S
    cases = [(512, 200.0), (1024, 100.0), (256, 50.0), (2048, 200.0)]
    fields = [shelf_fields(n, L, i) for i, (n, L) in enumerate(cases)]
    hxs = [O.deriv(h, L) for (h, _, _), (n, L) in zip(fields, cases)]
    bs = [O.apply_G_1d(e, hx, u, L) for (h, e, u), hx, (n, L) in zip(fields, hxs, cases)]
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L in cases])
        x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        sgn.pcg(lay, dev(pack([f[1] for f in fields])), dev(pack(hxs)), dev(pack(bs)), x,
                rtol=1e-10, prec=prec)
        xb = unpack(host(x), lay.offsets)
        for i, (n, L) in enumerate(cases):
            l1 = sgn.Layout(ctx, [sgn.Grid(1, n, L)])
            x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
            sgn.pcg(l1, dev(fields[i][1]), dev(hxs[i]), dev(bs[i]), x1, rtol=1e-10, prec=prec)
            assert np.array_equal(host(x1), xb[i])
            assert rel(xb[i], fields[i][2]) < 1e-8


def test_pcg_edge_cases(S):
    sgn, ctx = S
    n = 128
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    x = dev(np.ones(n))
    info = sgn.pcg(lay, dev(eta), dev(hx), dev(np.zeros(n)), x)[0]
    assert info["iters"] == 0 and np.all(host(x) == 0.0)
    ref = np.linalg.solve(O.dense_G_1d(eta, hx, 1.0), b)
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        x = dev(ref)
        info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-9, prec=prec)[0]
        assert info["iters"] == 0
    # maxit too small: reported, not silent
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-14, maxit=2, check=False)[0]
    assert info["status"] == 5
    with pytest.raises(sgn.SgnError):
        sgn.Layout(ctx, [sgn.Grid(1, 98, 1.0)])          # 2 7^2: no transform for radix 7


def test_rhs_shelf_and_flat(S):
    sgn, ctx = S
    cases = [(512, 200.0, 0), (4096, 200.0, 1), (256, 100.0, 2), (8192, 200.0, 3)]
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
        # F holds third derivatives: float64 rounding is amplified ~k_max^3.  The bound is
        # the oracle's own change under a last-bit relative perturbation of its inputs.
        rng = np.random.default_rng(i)
        jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.size))
        pe, pU = O.rhs_1d(jig(etas[i]), jig(us[i]), hs[i], jig(hxs[i]), L, 9.81)
        tol_e = max(1e-13, 20 * rel(pe, re))
        tol_U = max(1e-13, 20 * rel(pU, rU))
        assert rel(unpack(host(fe), lay.offsets)[i], re) < tol_e, (n, tol_e)
        assert rel(unpack(host(fU), lay.offsets)[i], rU) < tol_U, (n, tol_U)
        assert tol_U < 5e-9


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


def _run_oracle(c, scheme, nsteps, rtol, order=4):
    grid = O.make_grid(1, c.n, c.L, c.g)
    st = O.init_state(c.eta, c.u, c.h, grid)
    if scheme == "rk4":
        O.run_rk4(st, c.dt, nsteps, rtol)
    elif scheme == "ab":
        O.run_ab(st, order, c.dt, nsteps, rtol)
    else:
        O.run_sbdf2(st, c.dt, nsteps, rtol)
    return st


def test_rk4_solitary_wave_fp64_matches_oracle_and_closed_form(S):
    sgn, ctx = S
    c = I.solitary_case()                       # L=100, n=256, a=0.2, g=9.81, dt=0.01
    (eta, U, u), stats = _run_gpu(sgn, ctx, [c], "rk4", 40, "fp64", 1e-12)
    ref = _run_oracle(c, "rk4", 40, 1e-13)
    assert rel(eta[0], ref.eta) < 1e-11 and rel(u[0], ref.u) < 1e-10
    x = I.grid_1d(c.n, c.L)
    ee, ue = I.solitary_wave_1d(x, c.L, 1.0, 0.2, 25.0, c.g, t=0.4)
    assert np.abs(eta[0] - ee).max() < 1e-8
    assert stats["status"] == 0 and stats["solves"] == 40 * 4


@pytest.mark.parametrize("scheme,order", [("rk4", 0), ("ab", 2), ("ab", 3), ("ab", 4),
                                          ("linimp", 0)])
def test_steppers_shelf_fp64_match_oracle(S, scheme, order):
    sgn, ctx = S
    c = I.shelf_case(n=512, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = _run_gpu(sgn, ctx, [c], scheme, 25, "fp64", 1e-13, order or 4)
    ref = _run_oracle(c, scheme, 25, 1e-13, order or 4)
    zeta_ref = ref.eta - c.h
    assert rel(eta[0] - c.h, zeta_ref) < 1e-10
    assert rel(u[0], ref.u) < 1e-10
    assert rel(U[0], ref.U) < 1e-10


def test_rk4_mixed_precision_within_1e6(S):
    sgn, ctx = S
    c = I.shelf_case(n=1024, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = _run_gpu(sgn, ctx, [c], "rk4", 50, "mixed", 1e-11)
    ref = _run_oracle(c, "rk4", 50, 1e-13)
    assert rel(eta[0], ref.eta) < 1e-6 and rel(u[0], ref.u) < 1e-6
    assert stats["status"] == 0


def test_ensemble_batch_equals_alone(S):
    """Batched RK4 over uneven instances equals each instance advanced alone (bitwise)."""
    sgn, ctx = S
    ens = I.ensemble_1d(count=6, seed=7, kmin=9, kmax=11)
    (eta_b, _, u_b), _ = _run_gpu(sgn, ctx, ens, "rk4", 3, "mixed", 1e-10)
    for i, c in enumerate(ens):
        (eta_1, _, u_1), _ = _run_gpu(sgn, ctx, [c], "rk4", 3, "mixed", 1e-10)
        assert np.array_equal(eta_b[i], eta_1[0]) and np.array_equal(u_b[i], u_1[0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rk4_graph_replay_equals_direct_launches(S, prec):
    """From the second 1d RK4 step with unchanged options the library replays a captured CUDA
    graph of the step.  Alternating max_refine (12, 13: a cap never reached here) changes the
    options every call, which keeps every step on direct launches; both runs must agree
    bitwise, and so must the solver counters."""
    sgn, ctx = S
    ens = I.ensemble_1d(count=5, seed=11, kmin=8, kmax=11)
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    outs = []
    for alternate in (False, True):
        lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in ens])
        eta = dev(pack([c.eta for c in ens]))
        u = dev(pack([c.u for c in ens]))
        h = dev(pack([c.h for c in ens]))
        U = torch.zeros_like(eta)
        gh = torch.zeros_like(eta)
        st = sgn.State(lay, eta, U, u, h, gh)
        st.init()
        dts = [c.dt for c in ens]
        for k in range(5):
            mr = (12 + k % 2) if alternate else 12
            st.rk4(dts, 1, rtol=1e-10, prec=p, max_refine=mr)
        stats = st.stats()
        outs.append((host(eta), host(u), stats["iterations"], stats["solves"], stats["t"]))
        st.close()
        lay.close()
    (ea, ua, ia, sa, ta), (eb, ub, ib, sb, tb) = outs
    assert np.array_equal(ea, eb) and np.array_equal(ua, ub)
    assert (ia, sa) == (ib, sb) and ta == tb


def test_sbdf2_guard_counts_levels_past_the_fixed_A(S):
    """SBDF2 keeps the A of the initial data (§6.5); the state counts the instance-steps
    whose eta_max has grown past (4/3)^(1/3) of the initial one (the zero-stability bound of
    §5.4 for the generalised eigenvalues).  A shelf run stays clear of it; a depth raised by
    20% after init (ratio^3 = 1.73) is counted at every SBDF2 step."""
    sgn, ctx = S
    c = I.shelf_case(n=512, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g), sgn.Grid(1, 256, 100.0, g=9.81)])
    s2 = I.solitary_case()
    for scale, want in ((1.0, 0), (1.2, 5)):
        eta = dev(pack([c.eta, s2.eta]))
        u = dev(pack([c.u, s2.u]))
        h = dev(pack([c.h, s2.h]))
        U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
        st = sgn.State(lay, eta, U, u, h, gh)
        st.init()
        if scale != 1.0:
            eta[:c.n] *= scale                 # instance 0 only; A stays the initial one
        st.linimp([c.dt, s2.dt], 6, rtol=1e-12, maxit=4000, prec=sgn.PREC_FP64)
        stats = st.stats()
        st.close()
        # six steps: one RK4 start-up step, then five SBDF2 steps, each checked
        assert stats["sbdf2_stability_warnings"] == want, (scale, stats)


def test_pcg_async_writes_device_info_after_event(S):
    """sgn_pcg_async: the solve of sgn_pcg whose report lands in device memory; read after an
    event recorded on the stream, it equals sgn_pcg's report and the oracle's solution."""
    sgn, ctx = S
    cases = [(512, 1.0, 1.0), (2048, 4.0, 1.0), (8192, 1.0, 4.0)]
    prob = [I.testproblem_1d(n, e0, hv) for n, e0, hv in cases]
    hxs = [O.deriv(p[1], 1.0) for p in prob]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0) for n, _, _ in cases])
    eta, hx, b = dev(pack([p[2] for p in prob])), dev(pack(hxs)), dev(pack([p[3] for p in prob]))
    for prec, rtol, tol in ((sgn.PREC_FP64, 1e-12, 1e-10), (sgn.PREC_MIXED, 1e-11, 1e-9)):
        x_ref = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        info_ref = sgn.pcg(lay, eta, hx, b, x_ref, rtol=rtol, maxit=5000, prec=prec)
        s = torch.cuda.Stream()
        x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        info_dev = torch.full((len(cases) * sgn.PCG_INFO_BYTES,), 255, dtype=torch.uint8,
                              device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            sgn.pcg_async(lay, eta, hx, b, x, info_dev, rtol=rtol, maxit=5000, prec=prec,
                          stream=s)
            done = torch.cuda.Event()
            done.record(s)
        done.synchronize()
        info = sgn.pcg_info_from_bytes(bytes(info_dev.cpu().numpy().tobytes()), len(cases))
        assert info == info_ref
        xs = unpack(x.cpu().numpy(), lay.offsets)
        assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
        for i, (n, _, _) in enumerate(cases):
            assert info[i]["status"] == 0 and info[i]["ratio"] <= rtol
            ref = O.solve_G(prob[i][2], hxs[i], prob[i][3], O.make_grid(1, n, 1.0, 1.0),
                            rtol=1e-14, maxit=5000)[0]
            assert rel(xs[i], ref) < tol
    # a breakdown-free failure is reported through the device record, not the return value
    x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    info_dev = torch.zeros((len(cases) * sgn.PCG_INFO_BYTES,), dtype=torch.uint8, device="cuda")
    sgn.pcg_async(lay, eta, hx, b, x, info_dev, rtol=1e-14, maxit=2, prec=sgn.PREC_FP64)
    torch.cuda.synchronize()
    info = sgn.pcg_info_from_bytes(bytes(info_dev.cpu().numpy().tobytes()), len(cases))
    assert all(i["status"] == 5 for i in info)
