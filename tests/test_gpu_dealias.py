"""2/3-rule dealiasing of 1d and 2d states (sgn_state_set_dealias) against the oracle's.

Every new time level has its modes |j| > n/3 of zeta = eta - h and U removed before u is
solved from it (and of u too in SBDF2).  The steppers with dealiasing match the oracle's
dealiased steppers step for step (float64 1e-10, as the plain steppers in test_gpu_1d.py),
new levels carry no energy above n/3, and the dealiased SBDF2 run of the shelf at
dt = 0.002, which overflows without dealiasing before t = 8, reaches t = 8.
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


def top_energy(f):
    """Largest Fourier coefficient above n/3, relative to the largest overall."""
    n = f.size
    c = np.abs(np.fft.fft(f))
    j = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    return float(c[j > n / 3.0].max() / c.max())


def run_gpu(sgn, ctx, insts, scheme, plan, prec, rtol):
    """plan = [(dealias on?, steps), ...] applied in order on one state."""
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    eta, u, h = dev(pack([c.eta for c in insts])), dev(pack([c.u for c in insts])), \
        dev(pack([c.h for c in insts]))
    U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    dts = [c.dt for c in insts]
    for on, k in plan:
        st.set_dealias(on)
        if scheme == "rk4":
            st.rk4(dts, k, rtol=rtol, maxit=4000, prec=prec)
        elif scheme == "ab4":
            st.abk(4, dts, k, rtol=rtol, maxit=4000, prec=prec)
        else:
            st.linimp(dts, k, rtol=rtol, maxit=4000, prec=prec)
    stats = st.stats()
    out = [unpack(host(t), lay.offsets) for t in (eta, U, u)]
    st.close()
    return out, stats


def run_oracle(c, scheme, plan, rtol=1e-13):
    st = O.init_state(c.eta, c.u, c.h, O.make_grid(1, c.n, c.L, c.g))
    for on, k in plan:
        st.dealias = on
        if scheme == "rk4":
            O.run_rk4(st, c.dt, k, rtol)
        elif scheme == "ab4":
            O.run_ab(st, 4, c.dt, k, rtol)
        else:
            O.run_sbdf2(st, c.dt, k, rtol)
    return st


@pytest.mark.parametrize("scheme", ["rk4", "ab4", "sbdf2"])
def test_dealiased_steppers_match_oracle(S, scheme):
    sgn, ctx = S
    c = I.shelf_case(n=512, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = run_gpu(sgn, ctx, [c], scheme, [(True, 25)], sgn.PREC_FP64, 1e-13)
    ref = run_oracle(c, scheme, [(True, 25)])
    assert stats["status"] == 0
    assert rel(eta[0] - c.h, ref.eta - c.h) < 1e-10
    assert rel(u[0], ref.u) < 1e-10 and rel(U[0], ref.U) < 1e-10
    assert top_energy(eta[0] - c.h) < 1e-13 and top_energy(U[0]) < 1e-13
    if scheme == "sbdf2":
        assert top_energy(u[0]) < 1e-13
    # the projection changed the run: without it the state keeps its top modes
    plain = run_oracle(c, scheme, [(False, 25)])
    assert rel(plain.eta - c.h, ref.eta - c.h) > 1e-12


def test_dealias_ragged_batch_and_switching(S):
    """Every size class (one-CTA sizes, the clusters' n = 16384 with its global transform
    buffer) in one layout; dealiasing switched on after two plain RK4 steps, which also
    replaces the captured step graph."""
    sgn, ctx = S
    insts = [I.shelf_case(n=n, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0,
                          dt=0.25 * (200.0 / n) / np.sqrt(9.81 * 1.3))
             for n in (64, 1024, 8192, 16384)]
    for c in insts:
        c.dt = insts[-1].dt                          # one dt: the plan is per state
    plan = [(False, 2), (True, 2)]
    (eta, U, u), stats = run_gpu(sgn, ctx, insts, "rk4", plan, sgn.PREC_FP64, 1e-13)
    assert stats["status"] == 0
    for i, c in enumerate(insts):
        ref = run_oracle(c, "rk4", plan)
        assert rel(eta[i] - c.h, ref.eta - c.h) < 1e-10, c.n
        assert rel(u[i], ref.u) < 1e-10 and rel(U[i], ref.U) < 1e-10, c.n
        assert top_energy(eta[i] - c.h) < 1e-13 and top_energy(U[i]) < 1e-13, c.n


def test_dealiased_sbdf2_shelf_reaches_t8(S):
    """The shelf (N = 4096) with SBDF2 at dt = 0.002 for 4000 steps: without dealiasing the
    modes above n/3 grow (5e-11 at t = 6, 2e-8 at t = 7 in the oracle) and the run overflows
    before t = 8; with it, the mixed GPU run stays bounded to t = 8, within 1e-6 of the
    oracle's dealiased float64 run, and its crest (0.3697 in the oracle) agrees with AB4's
    at t = 8 (0.3695) to the schemes' time-discretisation error."""
    sgn, ctx = S
    c = I.shelf_case()
    c.dt = 0.002
    (eta, U, u), stats = run_gpu(sgn, ctx, [c], "sbdf2", [(True, 4000)], sgn.PREC_MIXED, 1e-12)
    z = eta[0] - c.h
    assert stats["status"] == 0 and np.isfinite(z).all() and abs(stats["t"] - 8.0) < 1e-9
    assert abs(np.abs(z).max() - 0.3695) < 2e-3
    assert top_energy(z) < 1e-13
    ref = run_oracle(c, "sbdf2", [(True, 4000)])
    assert rel(z, ref.eta - c.h) < 1e-6 and rel(u[0], ref.u) < 1e-6


def top_energy_2d(f):
    """Largest 2d Fourier coefficient outside |jx| <= nx/3, |jy| <= ny/3, relative to the
    largest overall; a vector field [2, ny, nx] counts its components together (they share
    one complex transform, hence one absolute rounding level)."""
    f = f if f.ndim == 3 else f[None]
    ny, nx = f.shape[1:]
    c = np.abs(np.fft.fft2(f, axes=(1, 2)))
    jx = np.abs(np.fft.fftfreq(nx, d=1.0 / nx))
    jy = np.abs(np.fft.fftfreq(ny, d=1.0 / ny))
    out = (jy[:, None] > ny / 3.0) | (jx[None, :] > nx / 3.0)
    return float(c[:, out].max() / c.max())


@pytest.mark.parametrize("scheme", ["rk4", "ab2", "sbdf2"])
def test_dealiased_2d_steppers_match_oracle(S, scheme):
    """2d: the tensor-product projection on the bump (32^2, 6 steps, float64)."""
    sgn, ctx = S
    c = I.bump2d_case(n=32, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
    n = c["n"]
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, c["L"], g=c["g"], ny=n, Ly=c["L"])])
    eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
    U, gh = torch.zeros_like(u), torch.zeros_like(u)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    st.set_dealias(True)
    if scheme == "rk4":
        st.rk4(c["dt"], 6, rtol=1e-13, maxit=4000, prec=sgn.PREC_FP64)
    elif scheme == "ab2":
        st.abk(2, c["dt"], 6, rtol=1e-13, maxit=4000, prec=sgn.PREC_FP64)
    else:
        st.linimp(c["dt"], 6, rtol=1e-13, maxit=4000, prec=sgn.PREC_FP64)
    assert st.stats()["status"] == 0
    e, UU, uu = host(eta).reshape(n, n), host(U).reshape(2, n, n), host(u).reshape(2, n, n)
    st.close()
    ref = O.init_state(c["eta"], c["u"], c["h"], O.make_grid(2, n, c["L"], c["g"], ny=n,
                                                                Ly=c["L"]))
    ref.dealias = True
    if scheme == "rk4":
        O.run_rk4(ref, c["dt"], 6, 1e-13)
    elif scheme == "ab2":
        O.run_ab(ref, 2, c["dt"], 6, 1e-13)
    else:
        O.run_sbdf2(ref, c["dt"], 6, 1e-13)
    assert rel(e - c["h"], ref.eta - c["h"]) < 1e-10
    assert rel(uu, ref.u) < 1e-10 and rel(UU, ref.U) < 1e-10
    assert top_energy_2d(e - c["h"]) < 1e-13
    assert top_energy_2d(UU) < 1e-13


@pytest.mark.parametrize("dealias", [False, True])
def test_mixed_sbdf2_ragged_with_the_cluster_size(S, dealias):
    """The double-float SBDF2 kernel and the double-float projection on every transform
    path (shared memory up to n = 8192, the global buffer at n = 16384) against the oracle's
    float64 steps."""
    sgn, ctx = S
    dt = 0.25 * (200.0 / 16384) / np.sqrt(9.81 * 1.3)
    insts = [I.shelf_case(n=n, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=dt)
             for n in (1024, 8192, 16384)]
    (eta, U, u), stats = run_gpu(sgn, ctx, insts, "sbdf2", [(dealias, 6)], sgn.PREC_MIXED,
                                 1e-12)
    assert stats["status"] == 0
    for i, c in enumerate(insts):
        ref = run_oracle(c, "sbdf2", [(dealias, 6)])
        assert rel(eta[i] - c.h, ref.eta - c.h) < 1e-6 and rel(u[i], ref.u) < 1e-6, c.n
        if dealias:
            assert top_energy(eta[i] - c.h) < 1e-13 and top_energy(u[i]) < 1e-12, c.n
