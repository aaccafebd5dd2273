"""RK4 on the non-constraint form (sgn_step_rk4_nc, 1d and 2d) against the oracle's
rk4_nc_step.

Each stage's u_t solves G u_t = M with M the u_t-free terms of Eq:MomEq; GPU and oracle
take the same steps, so float64 runs agree to 1e-10 (as the constraint-form steppers in
test_gpu_1d.py) and mixed ones to 1e-6.
"""
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
    return torch.as_tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pack(arrs):
    return np.concatenate([np.asarray(a, dtype=np.float64) for a in arrs])


def unpack(v, offs):
    return [v[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]


def run_gpu(sgn, ctx, insts, plan, prec, rtol):
    """plan = [("nc" | "rk4", steps), ...] on one state; returns eta, U, u per instance."""
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    eta, u, h = (dev(pack([getattr(c, k) for c in insts])) for k in ("eta", "u", "h"))
    U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    dts = [c.dt for c in insts]
    for kind, k in plan:
        if kind == "nc":
            st.rk4_nc(dts, k, rtol=rtol, maxit=4000, prec=prec)
        else:
            st.rk4(dts, k, rtol=rtol, maxit=4000, prec=prec)
    stats = st.stats()
    out = [unpack(host(t), lay.offsets) for t in (eta, U, u)]
    st.close()
    return out, stats


def run_oracle(c, plan, rtol=1e-13):
    st = O.init_state(c.eta, c.u, c.h, O.make_grid(1, c.n, c.L, c.g))
    for kind, k in plan:
        if kind == "nc":
            O.run_rk4_nc(st, c.dt, k, rtol)
        else:
            O.run_rk4(st, c.dt, k, rtol)
    return st


def test_rk4_nc_shelf_fp64_matches_oracle(S):
    sgn, ctx = S
    c = I.shelf_case(n=512, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = run_gpu(sgn, ctx, [c], [("nc", 25)], sgn.PREC_FP64, 1e-13)
    ref = run_oracle(c, [("nc", 25)])
    assert stats["status"] == 0 and stats["solves"] == 100
    assert rel(eta[0] - c.h, ref.eta - c.h) < 1e-10
    assert rel(u[0], ref.u) < 1e-10 and rel(U[0], ref.U) < 1e-10


def test_rk4_nc_mixed_within_1e6(S):
    sgn, ctx = S
    c = I.shelf_case(n=1024, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = run_gpu(sgn, ctx, [c], [("nc", 20)], sgn.PREC_MIXED, 1e-11)
    ref = run_oracle(c, [("nc", 20)])
    assert stats["status"] == 0
    assert rel(eta[0] - c.h, ref.eta - c.h) < 1e-6 and rel(u[0], ref.u) < 1e-6


def test_rk4_nc_ragged_batch_then_constraint_form(S):
    """Every size class in one layout (n = 16384 on its clusters); three non-constraint
    steps, then two constraint-form steps from the refreshed U = G u."""
    sgn, ctx = S
    dt = 0.25 * (200.0 / 16384) / np.sqrt(9.81 * 1.3)
    insts = [I.shelf_case(n=n, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=dt)
             for n in (64, 1024, 8192, 16384)]
    plan = [("nc", 3), ("rk4", 2)]
    (eta, U, u), stats = run_gpu(sgn, ctx, insts, plan, sgn.PREC_FP64, 1e-13)
    assert stats["status"] == 0
    for i, c in enumerate(insts):
        ref = run_oracle(c, plan)
        assert rel(eta[i] - c.h, ref.eta - c.h) < 1e-10, c.n
        assert rel(u[i], ref.u) < 1e-10 and rel(U[i], ref.U) < 1e-10, c.n


def test_rk4_nc_solitary_wave_closed_form(S):
    sgn, ctx = S
    c = I.solitary_case()
    (eta, U, u), _ = run_gpu(sgn, ctx, [c], [("nc", 40)], sgn.PREC_FP64, 1e-12)
    x = I.grid_1d(c.n, c.L)
    ee, ue = I.solitary_wave_1d(x, c.L, 1.0, 0.2, 25.0, c.g, t=0.4)
    assert np.abs(eta[0] - ee).max() < 1e-8 and np.abs(u[0] - ue).max() < 2e-8


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_rk4_nc_2d_bump_matches_oracle(S, prec, tol):
    """2d: the bump (32^2 and a 64 x 32 grid), 5 steps, then 2 constraint-form steps."""
    sgn, ctx = S
    for nx, ny in ((32, 32), (64, 32)):
        c = I.bump2d_case(n=32, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
        if nx != ny:
            X, Y = I.grid_2d(nx, ny, 40.0, 20.0)
            h = I.gaussian_bump_2d(X, Y, 40.0, 20.0, 0.5, 3.0, 20.0, 10.0)
            e0, u0 = I.solitary_wave_2d(X, Y, 40.0, 20.0, 1.0, 0.2, 10.0, 9.81)
            c = dict(c, h=h, eta=h + (e0 - 1.0), u=u0)
        Ly = 40.0 if nx == ny else 20.0
        lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 40.0, g=9.81, ny=ny, Ly=Ly)])
        eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
        U, gh = torch.zeros_like(u), torch.zeros_like(u)
        st = sgn.State(lay, eta, U, u, h, gh)
        st.init()
        p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
        rtol = 1e-13 if prec == "fp64" else 1e-11
        st.rk4_nc(c["dt"], 5, rtol=rtol, maxit=4000, prec=p)
        st.rk4(c["dt"], 2, rtol=rtol, maxit=4000, prec=p)
        assert st.stats()["status"] == 0
        e, uu, UU = host(eta).reshape(ny, nx), host(u).reshape(2, ny, nx), \
            host(U).reshape(2, ny, nx)
        st.close()
        ref = O.init_state(c["eta"], c["u"], c["h"], O.make_grid(2, nx, 40.0, 9.81, ny=ny, Ly=Ly))
        O.run_rk4_nc(ref, c["dt"], 5, 1e-13)
        O.run_rk4(ref, c["dt"], 2, 1e-13)
        assert rel(e - c["h"], ref.eta - c["h"]) < tol and rel(uu, ref.u) < tol, (nx, ny)
        assert rel(UU, ref.U) < tol, (nx, ny)


def test_rk4_nc_rejects_what_it_does_not_cover(S):
    sgn, ctx = S
    c = I.solitary_case(n=64, L=20.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g)])
    eta, u, h = dev(c.eta), dev(c.u), dev(c.h)
    st = sgn.State(lay, eta, torch.zeros_like(eta), u, h, torch.zeros_like(eta))
    st.init()
    st.set_dealias(True)
    with pytest.raises(sgn.SgnError):
        st.rk4_nc(0.01, 1)
    st.set_dealias(False)
    st.set_forcing(dev(np.zeros(64)), dev(np.zeros(64)), [1.0], [0.0])
    with pytest.raises(sgn.SgnError):
        st.rk4_nc(0.01, 1)
    st.set_forcing(None, None, [], [])
    st.rk4_nc(0.01, 1)
    st.close()
