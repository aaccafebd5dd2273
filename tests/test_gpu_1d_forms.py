"""Kernel forms of 1d size classes (sgn_layout_set_form / _get_form, sgn_state_autotune).

n = 4096 and 8192 can run on one CTA per instance or on two-CTA clusters.  The cluster
form must match the oracle as the one-CTA form does, the autotuner (sgn_state_autotune)
must pick valid forms, leave them in force and leave the state untouched, and a state's
captured step graph must follow a change of form.
Tolerances as in test_gpu_1d.py.
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
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pack(arrs):
    return np.concatenate([np.asarray(a, dtype=np.float64) for a in arrs])


def unpack(v, offs):
    return [v[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]


def shelf_fields(n, L, seed):
    rng = np.random.default_rng(seed)
    x = I.grid_1d(n, L)
    h = I.shelf_1d(x, L, r=0.5 + 0.2 * rng.random(), xs=0.3 * L, w=max(L / 40, 2 * L / n))
    eta = h + 0.2 * np.exp(-((x - 0.6 * L) / (0.05 * L)) ** 2)
    u = 0.3 * np.sin(2 * np.pi * x / L) + 0.05 * np.cos(6 * np.pi * x / L)
    return h, eta, u


@pytest.mark.parametrize("log2n", [12, 13])
def test_cluster_form_matches_oracle(S, log2n):
    """Solve (float64 and mixed) and right-hand side of the two-CTA form against the oracle,
    in a layout that mixes the class with one-CTA sizes."""
    sgn, ctx = S
    n = 1 << log2n
    cases = [(n, 200.0), (512, 3.0), (n, 100.0)]
    lay = sgn.Layout(ctx, [sgn.Grid(1, m, L, g=9.81) for m, L in cases])
    assert lay.form(log2n) == 1
    lay.set_form(log2n, 2)
    assert lay.form(log2n) == 2
    fields = [shelf_fields(m, L, i) for i, (m, L) in enumerate(cases)]
    hxs = [O.deriv(h, L) for (h, _, _), (m, L) in zip(fields, cases)]
    bs = [O.apply_G_1d(e, hx, u, L) for (h, e, u), hx, (m, L) in zip(fields, hxs, cases)]
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(pack([f[1] for f in fields])), dev(pack(hxs)), dev(pack(bs)), x,
                       rtol=1e-11, prec=prec)
        for i, (m, L) in enumerate(cases):
            assert info[i]["status"] == 0 and info[i]["ratio"] <= 1e-11
            ref, _, _, _ = O.solve_G(fields[i][1], hxs[i], bs[i], O.make_grid(1, m, L, 9.81),
                                     rtol=1e-14, maxit=5000)
            assert rel(unpack(host(x), lay.offsets)[i], ref) < 1e-9, (prec, m)
    fe = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    fU = torch.zeros_like(fe)
    sgn.rhs(lay, dev(pack([f[1] for f in fields])), dev(pack([f[2] for f in fields])),
            dev(pack([f[0] for f in fields])), dev(pack(hxs)), fe, fU)
    for i, (m, L) in enumerate(cases):
        h, eta, u = fields[i]
        re, rU = O.rhs_1d(eta, u, h, hxs[i], L, 9.81)
        rng = np.random.default_rng(i)
        jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.size))
        pe, pU = O.rhs_1d(jig(eta), jig(u), h, jig(hxs[i]), L, 9.81)
        assert rel(unpack(host(fe), lay.offsets)[i], re) < max(1e-13, 20 * rel(pe, re))
        assert rel(unpack(host(fU), lay.offsets)[i], rU) < max(1e-13, 20 * rel(pU, rU))


@pytest.mark.parametrize("solve_ctas,rhs_ctas", [(1, 2), (2, 1)])
def test_mixed_forms_rk4_match_oracle(S, solve_ctas, rhs_ctas):
    """Solve and right-hand side on different forms (the solve's u_x hand-off crosses from
    one form to the other): RK4 on n = 4096 and 8192 instances against the oracle."""
    sgn, ctx = S
    insts = [I.shelf_case(n=n, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0,
                          dt=0.25 * (200.0 / n) / np.sqrt(9.81 * 1.3)) for n in (4096, 8192)]
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    for l2 in (12, 13):
        lay.set_forms(l2, solve_ctas, rhs_ctas)
        assert lay.forms(l2) == (solve_ctas, rhs_ctas) and lay.form(l2) == solve_ctas
    eta = dev(pack([c.eta for c in insts]))
    u = dev(pack([c.u for c in insts]))
    h = dev(pack([c.h for c in insts]))
    U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    for prec, tol in ((sgn.PREC_FP64, 1e-9), (sgn.PREC_MIXED, 1e-6)):
        eta.copy_(dev(pack([c.eta for c in insts])))
        u.copy_(dev(pack([c.u for c in insts])))
        st.init()
        st.rk4([c.dt for c in insts], 3, rtol=1e-11 if prec == sgn.PREC_MIXED else 1e-13,
               maxit=4000, prec=prec)
        he, hu = unpack(host(eta), lay.offsets), unpack(host(u), lay.offsets)
        for i, c in enumerate(insts):
            ref = O.init_state(c.eta, c.u, c.h, O.make_grid(1, c.n, c.L, c.g))
            O.run_rk4(ref, c.dt, 3, 1e-13)
            assert rel(he[i] - c.h, ref.eta - c.h) < tol and rel(hu[i], ref.u) < tol, (prec, c.n)
    st.close()


def _rk4(sgn, ctx, insts, forms, plan, prec):
    """RK4 on a fresh state; plan = [(forms to set, steps), ...] applied in order."""
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    for l2, f in forms.items():
        lay.set_form(l2, f)
    eta = dev(pack([c.eta for c in insts]))
    u = dev(pack([c.u for c in insts]))
    h = dev(pack([c.h for c in insts]))
    U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    for fs, k in plan:
        for l2, f in fs.items():
            lay.set_form(l2, f)
        st.rk4([c.dt for c in insts], k, rtol=1e-11, maxit=4000, prec=prec)
    out = unpack(host(eta), lay.offsets), unpack(host(u), lay.offsets)
    st.close()
    return out


def test_cluster_form_rk4_matches_oracle_and_graph_follows_form_changes(S):
    sgn, ctx = S
    c = I.shelf_case(n=8192, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0,
                     dt=0.25 * (200.0 / 8192) / np.sqrt(9.81 * 1.3))
    ref = O.init_state(c.eta, c.u, c.h, O.make_grid(1, c.n, c.L, c.g))
    O.run_rk4(ref, c.dt, 3, 1e-13)
    (eta2, u2) = _rk4(sgn, ctx, [c], {13: 2}, [({}, 3)], sgn.PREC_FP64)
    assert rel(eta2[0] - c.h, ref.eta - c.h) < 1e-9 and rel(u2[0], ref.u) < 1e-9
    # the step graph is captured at the second step; a form change after it must be followed
    (eta_a, u_a) = _rk4(sgn, ctx, [c], {13: 1}, [({}, 2), ({13: 2}, 1)], sgn.PREC_MIXED)
    (eta_b, u_b) = _rk4(sgn, ctx, [c], {13: 1}, [({}, 3)], sgn.PREC_MIXED)
    assert not np.array_equal(u_a[0], u_b[0])          # the third step ran the cluster form
    assert rel(u_a[0], ref.u) < 1e-6 and rel(u_b[0], ref.u) < 1e-6


def test_autotune_on_a_state_keeps_valid_forms_and_restores_the_state(S):
    """sgn_state_autotune: times the forms on RK4 steps of the state's own problem, keeps a
    valid combination, and leaves the state as it found it: the run after tuning equals,
    bitwise, a run on a fresh layout with the same forms set by hand."""
    sgn, ctx = S
    ens = I.ensemble_1d(count=4, seed=11, kmin=12, kmax=13)
    dts = [c.dt for c in ens]

    def make(forms=None):
        lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in ens])
        for l2, (fs, fr) in (forms or {}).items():
            lay.set_forms(l2, fs, fr)
        eta = dev(pack([c.eta for c in ens]))
        u = dev(pack([c.u for c in ens]))
        h = dev(pack([c.h for c in ens]))
        U, gh = torch.zeros_like(eta), torch.zeros_like(eta)
        st = sgn.State(lay, eta, U, u, h, gh)
        st.init()
        return lay, st, (eta, U, u)

    lay, st, (eta, U, u) = make()
    before = [host(t).copy() for t in (eta, U, u)]
    ms = st.autotune(dts, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    assert ms > 0.0
    after = [host(t) for t in (eta, U, u)]
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    stats = st.stats()
    assert stats["solves"] == 0 and stats["step"] == 0 and stats["t"] == 0.0
    forms = {l2: lay.forms(l2) for l2 in (12, 13)}
    assert all(set(f) <= {1, 2} for f in forms.values())
    st.rk4(dts, 2, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    lay2, st2, (eta2, U2, u2) = make(forms)
    st2.rk4(dts, 2, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    assert torch.equal(u, u2) and torch.equal(eta, eta2) and torch.equal(U, U2)
    st.close()
    st2.close()


def test_set_form_arguments(S):
    sgn, ctx = S
    lay = sgn.Layout(ctx, [sgn.Grid(1, 2048, 1.0), sgn.Grid(1, 16384, 1.0)])
    with pytest.raises(sgn.SgnError) as e:
        lay.set_form(11, 2)                                 # no cluster form below 4096
    assert e.value.status == 2
    with pytest.raises(sgn.SgnError) as e:
        lay.set_form(14, 1)                                 # 16384 needs two CTAs
    assert e.value.status == 2
    with pytest.raises(sgn.SgnError) as e:
        lay.set_form(13, 3)
    assert e.value.status == 1
    with pytest.raises(sgn.SgnError) as e:
        lay.set_forms(14, 2, 1)                             # 16384's right-hand side too
    assert e.value.status == 2
    with pytest.raises(sgn.SgnError) as e:
        lay.set_forms(11, 1, 2)
    assert e.value.status == 2
    assert lay.form(14) == 2 and lay.form(11) == 1
    lay2 = sgn.Layout(ctx, [sgn.Grid(2, 32, 1.0, ny=32, Ly=1.0)])
    with pytest.raises(sgn.SgnError):
        lay2.set_form(12, 2)
