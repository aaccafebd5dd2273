"""Serving: continuous batching through sgn_batch_submit / poll / release.

Checks that requests arriving while others run are admitted and finish, that every result
equals the same request run alone through the direct API (bitwise for the batched 1d RK4
runs and 1d solves, whose instances own their CTAs), that oversize requests are rejected
against the memory budget, and that the timestamps are ordered.
"""
import time

import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_2506_16045_gb300 import sgn
    ctx = sgn.Context(0)
    yield sgn, ctx
    ctx.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serving requests did not finish"
        time.sleep(0.002)
    return out


def alone_run(sgn, ctx, c, scheme, nsteps, rtol, prec):
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g)])
    eta, u, h = dev(c.eta), dev(c.u), dev(c.h)
    U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    if scheme == sgn.SCHEME_RK4:
        st.rk4(c.dt, nsteps, rtol=rtol, maxit=4000, prec=prec)
    elif scheme == sgn.SCHEME_LINIMP:
        st.linimp(c.dt, nsteps, rtol=rtol, maxit=4000, prec=prec)
    else:
        st.abk(scheme, c.dt, nsteps, rtol=rtol, maxit=4000, prec=prec)
    torch.cuda.synchronize()
    res = eta.cpu().numpy(), u.cpu().numpy(), U.cpu().numpy()
    st.close()
    return res


def test_mixed_stream_results_equal_alone(S):
    sgn, ctx = S
    srv = sgn.Server(ctx)
    rtol, prec = 1e-10, sgn.PREC_MIXED
    ens = I.ensemble_1d(count=5, seed=11, kmin=9, kmax=12)
    steps = [3, 7, 20, 5, 12]
    # first wave
    tickets, spec = [], {}
    for c, k in zip(ens[:3], steps[:3]):
        st, t = srv.submit(sgn.REQ_RUN, sgn.Grid(1, c.n, c.L, g=c.g), dev(c.eta), dev(c.u),
                           dev(c.h), scheme=sgn.SCHEME_RK4, dt=c.dt, nsteps=k, rtol=rtol,
                           prec=prec)
        assert st == 0
        tickets.append(t)
        spec[t] = ("rk4", c, k)
    # 1d solves (Eq:Testproblem; n = 16384 on two-CTA clusters) and a multistep run,
    # submitted while the first wave runs
    for n in (256, 1024, 16384):
        _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
        st, t = srv.submit(sgn.REQ_SOLVE, sgn.Grid(1, n, 1.0), dev(eta), dev(b), dev(h),
                           rtol=1e-12, prec=prec, host=False)
        assert st == 0
        tickets.append(t)
        spec[t] = ("solve", (n, h, eta, b), None)
    c = ens[3]
    st, t = srv.submit(sgn.REQ_RUN, sgn.Grid(1, c.n, c.L, g=c.g), c.eta, c.u, c.h,
                       scheme=sgn.SCHEME_AB4, dt=c.dt, nsteps=steps[3], rtol=rtol, prec=prec,
                       host=True)
    assert st == 0
    tickets.append(t)
    spec[t] = ("ab4", c, steps[3])
    c = ens[4]
    st, t = srv.submit(sgn.REQ_RUN, sgn.Grid(1, c.n, c.L, g=c.g), dev(c.eta), dev(c.u), dev(c.h),
                       scheme=sgn.SCHEME_RK4, dt=c.dt, nsteps=steps[4], rtol=rtol, prec=prec)
    tickets.append(t)
    spec[t] = ("rk4", c, steps[4])
    c = I.ensemble_1d(count=3, seed=11, kmin=13, kmax=14)[2]
    assert c.n == 16384
    st, t = srv.submit(sgn.REQ_RUN, sgn.Grid(1, c.n, c.L, g=c.g), dev(c.eta), dev(c.u), dev(c.h),
                       scheme=sgn.SCHEME_RK4, dt=c.dt, nsteps=4, rtol=rtol, prec=prec)
    assert st == 0
    tickets.append(t)
    spec[t] = ("rk4", c, 4)
    res = wait(srv, tickets)
    for t in tickets:
        r = res[t]
        assert r["status"] == 0
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        kind, c, k = spec[t]
        if kind == "solve":
            n, h, eta, b = c
            x = sgn.device_array(r["u"], n).cpu().numpy()
            lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
            gh = torch.zeros(n, dtype=torch.float64, device="cuda")
            sgn.spectral_grad(lay, dev(h), gh)
            xa = torch.zeros(n, dtype=torch.float64, device="cuda")
            sgn.pcg(lay, dev(eta), gh, dev(b), xa, rtol=1e-12, maxit=4000, prec=prec)
            assert np.array_equal(x, xa.cpu().numpy())
            ref, _, _, _ = O.solve_G(eta, O.deriv(h, 1.0), b, O.make_grid(1, n, 1.0, 1.0),
                                     rtol=1e-14, maxit=4000)
            assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
        else:
            scheme = sgn.SCHEME_RK4 if kind == "rk4" else sgn.SCHEME_AB4
            ea, ua, Ua = alone_run(sgn, ctx, c, scheme, k, rtol, prec)
            eg = sgn.device_array(r["eta"], c.n).cpu().numpy()
            ug = sgn.device_array(r["u"], c.n).cpu().numpy()
            Ug = sgn.device_array(r["U"], c.n).cpu().numpy()
            assert np.array_equal(eg, ea) and np.array_equal(ug, ua) and np.array_equal(Ug, Ua)
        assert srv.release(t) == 0
    srv.close()


def test_2d_requests_in_the_mix(S):
    sgn, ctx = S
    srv = sgn.Server(ctx)
    c2 = I.bump2d_case(n=32, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
    g2 = sgn.Grid(2, 32, 40.0, g=9.81, ny=32, Ly=40.0)
    st, t_run = srv.submit(sgn.REQ_RUN, g2, dev(c2["eta"]), dev(c2["u"]), dev(c2["h"]),
                           scheme=sgn.SCHEME_RK4, dt=0.05, nsteps=4, rtol=1e-11,
                           prec=sgn.PREC_MIXED)
    assert st == 0
    _, _, h, eta, rhs = I.elliptical_bump_2d(32, 1.0, 1.0)
    st, t_sol = srv.submit(sgn.REQ_SOLVE, sgn.Grid(2, 32, 1.0, ny=32, Ly=1.0), dev(eta),
                           dev(rhs), dev(h), rtol=1e-12, prec=sgn.PREC_MIXED)
    assert st == 0
    res = wait(srv, [t_run, t_sol])
    assert res[t_run]["status"] == 0 and res[t_sol]["status"] == 0
    x = sgn.device_array(res[t_sol]["u"], 2 * 32 * 32).cpu().numpy().reshape(2, 32, 32)
    gh = O.grad(h, (1.0, 1.0))
    ref, _, _, _ = O.solve_G(eta, gh, rhs, O.make_grid(2, 32, 1.0, 1.0, ny=32, Ly=1.0),
                             rtol=1e-14, maxit=4000)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
    grid = O.make_grid(2, 32, 40.0, 9.81, ny=32, Ly=40.0)
    ost = O.init_state(c2["eta"], c2["u"], c2["h"], grid)
    O.run_rk4(ost, 0.05, 4, 1e-13)
    eg = sgn.device_array(res[t_run]["eta"], 32 * 32).cpu().numpy().reshape(32, 32)
    assert np.linalg.norm(eg - ost.eta) / np.linalg.norm(ost.eta) < 1e-6
    for t in (t_run, t_sol):
        srv.release(t)
    srv.close()


def test_admission_budget_and_rejection(S):
    sgn, ctx = S
    free, total = torch.cuda.mem_get_info()
    # a budget that holds about one 2d 512^2 request: an oversize 1024^2 request is rejected
    frac = 1.5 * (5 * 8 * 512 * 512 + 816 * 512 * 512) / total
    srv = sgn.Server(ctx, budget_fraction=frac)
    z = torch.zeros(2 * 1024 * 1024, dtype=torch.float64, device="cuda")
    st, _ = srv.submit(sgn.REQ_SOLVE, sgn.Grid(2, 1024, 1.0, ny=1024, Ly=1.0), z, z, z)
    assert st == 10                                # SGN_ERR_REJECTED
    # several small requests still run to completion under the same budget
    tickets = []
    for n in (512, 1024, 2048):
        _, h, eta, b = I.testproblem_1d(n, 1.0, 0.5)
        st, t = srv.submit(sgn.REQ_SOLVE, sgn.Grid(1, n, 1.0), dev(eta), dev(b), dev(h),
                           rtol=1e-10)
        assert st == 0
        tickets.append(t)
    res = wait(srv, tickets)
    assert all(r["status"] == 0 for r in res.values())
    srv.close()


def test_short_solve_overlaps_a_long_2d_run(S):
    """Work of admitted requests overlaps on the device: a short 1d solve submitted while a
    2d run's chunk of steps is in flight finishes before that chunk, and the 2d run's result
    is bitwise the run alone."""
    sgn, ctx = S
    n2 = 512
    c2 = I.bump2d_case(n=n2, L=80.0, a=0.2, x0=20.0, H=0.5, R=3.0, dt=0.02)
    g2 = sgn.Grid(2, n2, 80.0, g=9.81, ny=n2, Ly=80.0)
    nsteps = 16                                   # one chunk of the server
    srv = sgn.Server(ctx)
    st, t_run = srv.submit(sgn.REQ_RUN, g2, dev(c2["eta"]), dev(c2["u"]), dev(c2["h"]),
                           scheme=sgn.SCHEME_RK4, dt=0.02, nsteps=nsteps, rtol=1e-10,
                           prec=sgn.PREC_MIXED)
    assert st == 0
    time.sleep(0.03)                              # the chunk is on the device by now
    _, h, eta, b = I.testproblem_1d(1024, 1.0, 1.0)
    st, t_sol = srv.submit(sgn.REQ_SOLVE, sgn.Grid(1, 1024, 1.0), dev(eta), dev(b), dev(h),
                           rtol=1e-10, prec=sgn.PREC_MIXED)
    assert st == 0
    res = wait(srv, [t_run, t_sol])
    rr, rs = res[t_run], res[t_sol]
    assert rr["status"] == 0 and rs["status"] == 0
    # the solve was admitted and finished while the run's only chunk was still running
    assert rr["t_admit"] < rs["t_admit"] and rs["t_done"] < rr["t_done"], (rr, rs)
    # the 2d run equals the same run alone
    eta_a, u_a, h_a = dev(c2["eta"]), dev(c2["u"]), dev(c2["h"])
    U_a = torch.zeros(2 * n2 * n2, dtype=torch.float64, device="cuda")
    gh_a = torch.zeros_like(U_a)
    lay = sgn.Layout(ctx, [g2])
    sta = sgn.State(lay, eta_a, U_a, u_a, h_a, gh_a)
    sta.init()
    sta.rk4(0.02, nsteps, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    torch.cuda.synchronize()
    eg = sgn.device_array(rr["eta"], n2 * n2).cpu().numpy()
    ug = sgn.device_array(rr["u"], 2 * n2 * n2).cpu().numpy()
    assert np.array_equal(eg, eta_a.cpu().numpy()) and np.array_equal(ug, u_a.cpu().numpy())
    sta.close()
    for t in (t_run, t_sol):
        srv.release(t)
    srv.close()


def test_release_while_other_work_is_in_flight(S):
    """Results released as soon as they are done, while a 2d run keeps the server busy (so
    their working memory is still queued for the deferred frees): the server frees each
    request exactly once, a released ticket is gone, and later requests still finish."""
    sgn, ctx = S
    n2 = 256
    c2 = I.bump2d_case(n=n2, L=80.0, a=0.2, x0=20.0, H=0.5, R=3.0, dt=0.02)
    g2 = sgn.Grid(2, n2, 80.0, g=9.81, ny=n2, Ly=80.0)
    srv = sgn.Server(ctx)
    st, t_run = srv.submit(sgn.REQ_RUN, g2, dev(c2["eta"]), dev(c2["u"]), dev(c2["h"]),
                           scheme=sgn.SCHEME_RK4, dt=0.02, nsteps=48, rtol=1e-10,
                           prec=sgn.PREC_MIXED)
    assert st == 0
    for wave in range(3):
        tickets = []
        for n in (256, 512, 1024, 2048):
            _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
            st, t = srv.submit(sgn.REQ_SOLVE, sgn.Grid(1, n, 1.0), eta, b, h, rtol=1e-10,
                               prec=sgn.PREC_MIXED, host=True)
            assert st == 0
            tickets.append(t)
        res = wait(srv, tickets)
        for t in tickets:
            assert res[t]["status"] == 0
            assert srv.release(t) == 0
            assert srv.release(t) == 1                 # gone: SGN_ERR_INVALID_ARG
    res = wait(srv, [t_run])
    assert res[t_run]["status"] == 0
    srv.release(t_run)
    srv.close()


def test_2d_runs_and_solves_of_several_sizes(S):
    """2d solves and 2d runs of several grid sizes interleaved on the 2d lane (each request's
    layout builds its own solve graph while layouts of other sizes come and go): every
    request finishes with status 0 and every solve returns its known solution."""
    sgn, ctx = S
    srv = sgn.Server(ctx)
    sizes = [256, 64, 128, 32, 256, 64]
    tickets, known = [], {}
    for i, n in enumerate(sizes):
        c = I.bump2d_case(n=n, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05 * 64 / n)
        g2 = sgn.Grid(2, n, 40.0, g=9.81, ny=n, Ly=40.0)
        if i % 2 == 0:
            st, t = srv.submit(sgn.REQ_RUN, g2, dev(c["eta"]), dev(c["u"]), dev(c["h"]),
                               scheme=sgn.SCHEME_RK4, dt=0.05 * 64 / n, nsteps=20, rtol=1e-10,
                               prec=sgn.PREC_MIXED)
        else:
            gh = O.grad(c["h"], (40.0, 40.0))
            grid = O.make_grid(2, n, 40.0, 9.81, ny=n, Ly=40.0)
            b = O.apply_G(c["eta"], gh, c["u"], grid)
            st, t = srv.submit(sgn.REQ_SOLVE, g2, dev(c["eta"]), dev(b), dev(c["h"]),
                               rtol=1e-10, prec=sgn.PREC_MIXED)
            known[t] = (n, c["u"])
        assert st == 0
        tickets.append(t)
    res = wait(srv, tickets, timeout=300.0)
    for t in tickets:
        assert res[t]["status"] == 0, res[t]
        if t in known:
            n, u = known[t]
            x = sgn.device_array(res[t]["u"], 2 * n * n).cpu().numpy().reshape(2, n, n)
            assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-8
        srv.release(t)
    srv.close()


def test_generic_sizes_are_served(S):
    """Requests on sizes that are not powers of two (1d n = 384 and 1536, 2d 96 x 60) are
    admitted and finish, each equal to the same request run alone through the direct API."""
    sgn, ctx = S
    srv = sgn.Server(ctx)
    tickets, spec = [], {}
    for n in (384, 1536):
        _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
        st, t = srv.submit(sgn.REQ_SOLVE, sgn.Grid(1, n, 1.0), dev(eta), dev(b), dev(h),
                           rtol=1e-11, prec=sgn.PREC_MIXED)
        assert st == 0
        tickets.append(t)
        spec[t] = ("solve1", n, h, eta, b)
    c = I.ensemble_1d(count=1, seed=5, sizes=[768])[0]
    st, t = srv.submit(sgn.REQ_RUN, sgn.Grid(1, c.n, c.L, g=c.g), dev(c.eta), dev(c.u), dev(c.h),
                       scheme=sgn.SCHEME_RK4, dt=c.dt, nsteps=6, rtol=1e-10, prec=sgn.PREC_MIXED)
    assert st == 0
    tickets.append(t)
    spec[t] = ("run1", c)
    nx, ny, Lx, Ly = 96, 60, 24.0, 15.0
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    h2 = I.gaussian_bump_2d(X, Y, Lx, Ly, 0.4, 3.0, Lx / 2, Ly / 2)
    eta2 = h2 + 0.2 * np.exp(np.cos(2 * np.pi * X / Lx) - 1)
    us = np.stack([0.3 * np.sin(2 * np.pi * X / Lx), 0.2 * np.cos(2 * np.pi * Y / Ly)])
    grid = O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly)
    b2 = O.apply_G(eta2, O.grad(h2, (Lx, Ly)), us, grid)
    st, t = srv.submit(sgn.REQ_SOLVE, sgn.Grid(2, nx, Lx, g=9.81, ny=ny, Ly=Ly), dev(eta2),
                       dev(b2), dev(h2), rtol=1e-11, prec=sgn.PREC_MIXED)
    assert st == 0
    tickets.append(t)
    spec[t] = ("solve2", us)
    res = wait(srv, tickets)
    for t in tickets:
        r = res[t]
        assert r["status"] == 0, (spec[t][0], r)
        kind = spec[t][0]
        if kind == "solve1":
            _, n, h, eta, b = spec[t]
            x = sgn.device_array(r["u"], n).cpu().numpy()
            ref = O.solve_G(eta, O.deriv(h, 1.0), b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-14,
                            maxit=4000)[0]
            assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
        elif kind == "run1":
            c = spec[t][1]
            ea, ua, Ua = alone_run(sgn, ctx, c, sgn.SCHEME_RK4, 6, 1e-10, sgn.PREC_MIXED)
            eg = sgn.device_array(r["eta"], c.n).cpu().numpy()
            ug = sgn.device_array(r["u"], c.n).cpu().numpy()
            assert np.array_equal(eg, ea) and np.array_equal(ug, ua)
        else:
            x = sgn.device_array(r["u"], 2 * nx * ny).cpu().numpy().reshape(2, ny, nx)
            assert np.linalg.norm(x - spec[t][1]) / np.linalg.norm(spec[t][1]) < 1e-8
        srv.release(t)
    srv.close()
