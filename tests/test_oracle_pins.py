"""Pins of the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed form, a value
printed in the paper, a theorem of the paper, an invariant, or a second construction that
shares no code with the first.  A plausible slip in the oracle (a dropped term, a sign, a
transposed operand, a wrong coefficient) breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ---------------------------------------------------------------------------- D (§6.1)

@pytest.mark.parametrize("n,L", [(8, 1.0), (16, 3.7), (64, 100.0), (128, 2 * math.pi),
                                 (6, 1.0), (12, 2.0), (30, 5.0), (96, 80.0), (120, 1.5)])
def test_derivative_fft_equals_cotangent_matrix(n, L):
    """D built from the DFT definition equals the closed-form periodic cotangent matrix."""
    Df = O.diff_matrix_fft(n, L)
    Dc = O.diff_matrix_cot(n, L)
    assert np.abs(Df - Dc).max() <= 1e-14 * np.abs(Dc).max() * n
    assert np.abs(Dc + Dc.T).max() == 0.0           # real antisymmetric


@pytest.mark.parametrize("n,L", [(16, 1.0), (64, 7.5), (30, 2.0), (96, 7.5), (384, 80.0)])
def test_derivative_exact_on_trig_and_nyquist(n, L):
    x = I.grid_1d(n, L)
    for m in range(1, n // 2):
        f = np.sin(2 * np.pi * m * x / L)
        np.testing.assert_allclose(O.deriv(f, L), (2 * np.pi * m / L) * np.cos(2 * np.pi * m * x / L),
                                   atol=1e-12 * (2 * np.pi * m / L))
    nyq = np.cos(np.pi * n * x / L)                    # the n/2 mode: its derivative is 0 (§6.1)
    assert np.abs(O.deriv(nyq, L)).max() < 1e-12
    assert np.abs(O.deriv(np.ones(n), L)).max() < 1e-14


def test_derivative_2d_tensor_product():
    X, Y = I.grid_2d(16, 8, 2.0, 3.0)
    f = np.sin(2 * np.pi * 3 * X / 2.0) * np.cos(2 * np.pi * 2 * Y / 3.0)
    g = O.grad(f, (2.0, 3.0))
    np.testing.assert_allclose(g[0], (2 * np.pi * 3 / 2.0) * np.cos(2 * np.pi * 3 * X / 2.0)
                               * np.cos(2 * np.pi * 2 * Y / 3.0), atol=1e-12)
    np.testing.assert_allclose(g[1], -(2 * np.pi * 2 / 3.0) * np.sin(2 * np.pi * 3 * X / 2.0)
                               * np.sin(2 * np.pi * 2 * Y / 3.0), atol=1e-12)


# ---------------------------------------------------------------------------- G (Def:G)

@pytest.mark.parametrize("eta0,hvar", [(1.0, 1.0), (4.0, 0.5), (0.5, 4.0)])
def test_G_matrix_free_equals_dense_weak_form_1d(eta0, hvar):
    """Def:G term by term (FFT derivatives) equals W^T M W (Def:MatrixM, cotangent D)."""
    n = 48
    _, h, eta, _ = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0)
    Gd = O.dense_G_1d(eta, hx, 1.0)
    U = np.random.default_rng(3).standard_normal((n, 5))
    mf = np.stack([O.apply_G_1d(eta, hx, U[:, i], 1.0) for i in range(5)], axis=1)
    assert np.abs(Gd @ U - mf).max() <= 1e-13 * np.abs(Gd @ U).max()
    assert np.abs(Gd - Gd.T).max() <= 1e-14 * np.abs(Gd).max()
    np.linalg.cholesky(Gd)                              # SPD (§6.1)


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, 20.0)])
def test_G_matrix_free_equals_dense_weak_form_2d(a, b):
    n = 10
    _, _, h, eta, _ = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    Gd = O.dense_G_2d(eta, gh, 1.0, 1.0)
    u = np.random.default_rng(4).standard_normal((2, n, n))
    ref = Gd @ u.ravel()
    assert np.abs(ref - O.apply_G(eta, gh, u, grid).ravel()).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(Gd - Gd.T).max() <= 1e-14 * np.abs(Gd).max()
    np.linalg.cholesky(Gd)


def test_G_2d_reduces_to_1d_on_y_constant_fields():
    """§6.3: extending 1d data as constants in y with v = 0 reproduces the 1d operator."""
    n, ny = 32, 4
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    u1 = np.random.default_rng(5).standard_normal(n)
    g1 = O.apply_G_1d(eta, hx, u1, 1.0)
    E = np.tile(eta, (ny, 1))
    H = np.tile(h, (ny, 1))
    gh = O.grad(H, (1.0, 0.7))
    U2 = np.stack([np.tile(u1, (ny, 1)), np.zeros((ny, n))])
    g2 = O.apply_G(E, gh, U2, O.make_grid(2, n, 1.0, 1.0, ny=ny, Ly=0.7))
    np.testing.assert_allclose(g2[0], np.tile(g1, (ny, 1)), atol=1e-12 * np.abs(g1).max())
    assert np.abs(g2[1]).max() < 1e-12 * np.abs(g1).max()


def test_flat_constant_depth_gives_A_equal_G_and_one_iteration():
    """Eq:FlatbathCoeff with constant eta: A = G, kappa_ub = 1, PCG stops after 1 iteration."""
    n, L, eta0 = 64, 10.0, 1.7
    eta = np.full(n, eta0)
    hx = np.zeros(n)
    c = O.precond_coeffs(eta, hx)
    gold = GOLDEN["flat_optimality"]
    assert c["flat"] and c["kappa_ub"] == gold["kappa_ub"]
    assert c["sigma"] == eta0 and abs(c["alpha"] - eta0 ** 3 / 3) < 1e-15
    Gd = O.dense_G_1d(eta, hx, L)
    Ad = O.dense_A_1d(c["sigma"], c["alpha"], n, L)
    assert np.abs(Gd - Ad).max() <= 1e-13 * np.abs(Ad).max()
    b = np.random.default_rng(6).standard_normal(n)
    grid = O.make_grid(1, n, L, 9.81)
    x, it, ratio, _ = O.solve_G(eta, hx, b, grid, rtol=1e-12)
    assert it == gold["pcg_iterations"]
    np.testing.assert_allclose(Gd @ x, b, atol=1e-12 * np.abs(b).max())


# ---------------------------------------------------------------------------- A (Def:A)

def test_Ainv_inverts_dense_A_1d_and_2d():
    n, L = 32, 2.5
    r = np.random.default_rng(7).standard_normal(n)
    z = O.apply_Ainv(r, 1.3, 0.4, O.make_grid(1, n, L, 1.0))
    np.testing.assert_allclose(O.dense_A_1d(1.3, 0.4, n, L) @ z, r, atol=1e-12)
    nx, ny = 8, 6
    r2 = np.random.default_rng(8).standard_normal((2, ny, nx))
    grid = O.make_grid(2, nx, 1.5, 1.0, ny=ny, Ly=2.0)
    z2 = O.apply_Ainv(r2, 0.9, 0.3, grid)
    np.testing.assert_allclose(O.dense_A_2d(0.9, 0.3, nx, ny, 1.5, 2.0) @ z2.ravel(), r2.ravel(),
                               atol=1e-12)
    np.testing.assert_allclose(O.apply_A(z2, 0.9, 0.3, grid), r2, atol=1e-12)


# ---------------------------------------------------------------------------- Theorem 4.1

def test_lambda_pm_printed_values():
    gold = GOLDEN["lambda_pm"]
    ev = np.linalg.eigvalsh(np.array([[1.0, 0.5], [0.5, 1.0 / 3.0]]))
    assert abs(ev[1] - O.LAMBDA_PLUS) < 1e-15 and abs(ev[0] - O.LAMBDA_MINUS) < 1e-15
    assert abs(O.LAMBDA_PLUS - eval(gold["plus_formula"], {"sqrt": math.sqrt})) < 1e-15
    assert abs(O.LAMBDA_PLUS / O.LAMBDA_MINUS - 19.28147006790397) < 1e-12


@pytest.mark.parametrize("eta0", [0.5, 1.0, 4.0])
@pytest.mark.parametrize("hvar", [0.0, 0.5, 1.0, 4.0])
@pytest.mark.parametrize("n", [16, 64, 24, 40])
def test_theorem_4_1_eigenvalue_interval_1d(n, eta0, hvar):
    """Generalized eigenvalues of (G, A) lie in [1/kappa_ub, 1] (Eq:EigValueBound)."""
    _, h, eta, _ = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0) if hvar else np.zeros(n)
    c = O.precond_coeffs(eta, hx)
    ev = O.generalized_eigenvalues(O.dense_G_1d(eta, hx, 1.0),
                                   O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0))
    assert ev.min() >= (1.0 - 1e-12) / c["kappa_ub"]
    assert ev.max() <= 1.0 + 1e-12
    cr = O.precond_coeffs(eta, hx, "replacement")
    assert cr["kappa_ub"] >= c["kappa_ub"] * (1 - 1e-14)
    evr = O.generalized_eigenvalues(O.dense_G_1d(eta, hx, 1.0),
                                    O.dense_A_1d(cr["sigma"], cr["alpha"], n, 1.0))
    assert evr.min() >= (1.0 - 1e-12) / cr["kappa_ub"] and evr.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, 20.0)])
def test_theorem_4_1_eigenvalue_interval_2d(a, b):
    n = 12
    _, _, h, eta, _ = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    c = O.precond_coeffs(eta, gh)
    ev = O.generalized_eigenvalues(O.dense_G_2d(eta, gh, 1.0, 1.0),
                                   O.dense_A_2d(c["sigma"], c["alpha"], n, n, 1.0, 1.0))
    assert ev.min() >= (1.0 - 1e-12) / c["kappa_ub"]
    assert ev.max() <= 1.0 + 1e-12


def test_flat_bottom_coefficients_are_the_sharp_ones():
    """On a flat bottom the bound (eta_max/eta_min)^3 is attained up to discretisation."""
    n = 64
    _, _, eta, _ = I.testproblem_1d(n, 1.0, 0.0)
    hx = np.zeros(n)
    c = O.precond_coeffs(eta, hx)
    ev = O.generalized_eigenvalues(O.dense_G_1d(eta, hx, 1.0),
                                   O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0))
    assert abs(c["kappa_ub"] - 8.0) < 1e-12
    assert ev.max() > 0.95 and ev.min() < 1.2 / c["kappa_ub"]


def test_printed_testproblem_values():
    """|h_x|_max ~ 17.2 |h0| and the eigenvalue bulk ~[3e-2, 3e-1] with ~6 outliers (§6.2)."""
    g = GOLDEN["hx_max_testproblem"]
    assert abs(20 * math.sqrt(2) / math.exp(0.5) - g["exact"]) < 1e-12
    assert round(g["exact"], 1) == g["printed"]
    gb = GOLDEN["eigen_bulk_testproblem"]
    for n in gb["n"]:
        _, h, eta, _ = I.testproblem_1d(n, 1.0, 1.0)
        hx = O.deriv(h, 1.0)
        assert abs(np.abs(hx).max() - g["exact"]) < (0.3 if n == 64 else 1e-3)
        c = O.precond_coeffs(eta, hx)
        ev = O.generalized_eigenvalues(O.dense_G_1d(eta, hx, 1.0),
                                       O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0))
        outside = int(np.sum((ev < gb["bulk_lo"]) | (ev > gb["bulk_hi"])))
        assert 3 <= outside <= 10
        assert ev.min() >= 1.0 / c["kappa_ub"]


# ---------------------------------------------------------------------------- PCG (§3.2)

@pytest.mark.parametrize("eta0,hvar", [(1.0, 1.0), (4.0, 1.0)])
def test_pcg_error_monotone_and_within_cg_bound(eta0, hvar):
    """epsilon(u_j) is non-increasing (§6.1) and <= 2 rho^j epsilon(0) (Eq:pcg_upperbound)."""
    n = 64
    _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    Gd = O.dense_G_1d(eta, hx, 1.0)
    ustar = np.linalg.solve(Gd, b)
    c = O.precond_coeffs(eta, hx)
    x, it, ratio, hist = O.pcg(lambda v: O.apply_G(eta, hx, v, grid),
                               lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid),
                               b, None, 1e-13, 500, history=True)
    eps = [O.g_error(u, ustar, Gd, b) for u in hist]
    rho = (math.sqrt(c["kappa_ub"]) - 1) / (math.sqrt(c["kappa_ub"]) + 1)
    for j in range(1, len(eps)):
        assert eps[j] <= eps[j - 1] * (1 + 1e-9) + 1e-15
        assert eps[j] <= 2 * rho ** j * eps[0] * (1 + 1e-9) + 1e-15
    assert eps[-1] < 1e-12
    # reading R7: stopping at sqrt(r.A^-1 r) <= rtol sqrt(b.A^-1 b) gives
    # eps <= sqrt(kappa_ub) rtol sqrt(b.A^-1 b)/||b||, since G^-1 <= kappa_ub A^-1
    bAb = float(b @ O.apply_Ainv(b, c["sigma"], c["alpha"], grid))
    for rtol in (1e-4, 1e-7):
        x, _, _ = O.pcg(lambda v: O.apply_G(eta, hx, v, grid),
                        lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid), b, None, rtol, 500)
        bound = math.sqrt(c["kappa_ub"]) * rtol * math.sqrt(bAb) / np.linalg.norm(b)
        assert O.g_error(x, ustar, Gd, b) <= bound * 1.01


@pytest.mark.parametrize("eta0,hvar", [(1.0, 1.0), (4.0, 1.0), (1.0, 4.0)])
def test_pcg_iterations_bounded_under_mesh_refinement(eta0, hvar):
    """§6.2: the iterations grow with eta0 and h0 but stay bounded as n grows (the discrete
    bound kappa(A^{-1}G) <= kappa_ub holds at every n): from n = 1024 to 16384 the count to
    rtol 1e-12 changes by at most 2, and kappa_ub converges to its continuum value."""
    its, kap = [], []
    for n in (1024, 4096, 16384):
        _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
        hx = O.deriv(h, 1.0)
        _, it, ratio, c = O.solve_G(eta, hx, b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-12,
                                    maxit=5000)
        assert ratio <= 1e-12
        its.append(it), kap.append(c["kappa_ub"])
    assert max(its) - min(its) <= 2, its
    assert abs(kap[2] - kap[1]) <= 1e-3 * kap[2]
    rho = (math.sqrt(kap[2]) - 1) / (math.sqrt(kap[2]) + 1)
    assert its[2] <= math.log(1e-12 / 2) / math.log(rho)       # inside the CG bound's count


def test_replacement_coefficients_lose_only_where_eta_is_small_at_steep_bottom():
    """§6.2's comparison of sigma*, alpha* with the replacement coefficients on the square-wave
    depth: when eta is small where |h_x| is large (eta0 < 1 here) sigma** exceeds sigma* and
    PCG needs more iterations to epsilon < 1e-8 (def:discrete_Gerr); when the condition fails
    (eta0 = 5) the two coefficient sets give the same iteration count."""
    n = 256
    grid = O.make_grid(1, n, 1.0, 1.0)
    counts = {}
    for eta0 in (0.25, 5.0):
        _, h, eta, b = I.squarewave_1d(n, eta0)
        hx = O.deriv(h, 1.0)
        Gd = O.dense_G_1d(eta, hx, 1.0)
        ustar = np.linalg.solve(Gd, b)
        for kind in ("opt", "replacement"):
            c = O.precond_coeffs(eta, hx, kind)
            _, _, _, hist = O.pcg(lambda v: O.apply_G(eta, hx, v, grid),
                                  lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid),
                                  b, None, 1e-15, 400, history=True)
            eps = [O.g_error(u, ustar, Gd, b) for u in hist]
            counts[(eta0, kind)] = (next(j for j, e in enumerate(eps) if e < 1e-8), c["sigma"])
    (io, so), (ir, sr) = counts[(0.25, "opt")], counts[(0.25, "replacement")]
    assert sr > 1.5 * so and ir >= io + 10, counts
    (io, so), (ir, sr) = counts[(5.0, "opt")], counts[(5.0, "replacement")]
    assert abs(ir - io) <= 1, counts


def test_pcg_zero_rhs_and_exact_warm_start():
    n = 32
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    x, it, _, _ = O.solve_G(eta, hx, np.zeros(n), grid, x0=np.ones(n))
    assert it == 0 and np.all(x == 0)
    ustar = np.linalg.solve(O.dense_G_1d(eta, hx, 1.0), b)
    x, it, _, _ = O.solve_G(eta, hx, b, grid, x0=ustar, rtol=1e-10)
    assert it == 0


def test_pcg_2d_elliptical_bump_converges_to_dense_solution():
    n = 12
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, 1.0, 20.0)
    gh = O.grad(h, (1.0, 1.0))
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    x, it, ratio, c = O.solve_G(eta, gh, rhs, grid, rtol=1e-13)
    ref = np.linalg.solve(O.dense_G_2d(eta, gh, 1.0, 1.0), rhs.ravel())
    np.testing.assert_allclose(x.ravel(), ref, atol=1e-10 * np.abs(ref).max())


# ---------------------------------------------------------------------------- time stepping

def test_solitary_wave_closed_form_rk4():
    """Flat bottom, L=100, n=256, a=0.2, g=9.81: RK4 follows the exact translating wave."""
    case = I.solitary_case()
    grid = O.make_grid(1, case.n, case.L, case.g)
    st = O.init_state(case.eta, case.u, case.h, grid)
    O.run_rk4(st, 0.01, 60)
    x = I.grid_1d(case.n, case.L)
    ee, ue = I.solitary_wave_1d(x, case.L, 1.0, 0.2, 25.0, case.g, t=st.t)
    assert np.abs(st.eta - ee).max() < 1e-8
    assert np.abs(st.u - ue).max() < 1e-8


def _order_errors(run, dts, T=1.0):
    case = I.solitary_case(n=128, L=60.0, a=0.3, x0=30.0, g=1.0)
    x = I.grid_1d(case.n, case.L)
    errs = []
    for dt in dts:
        grid = O.make_grid(1, case.n, case.L, case.g)
        st = O.init_state(case.eta, case.u, case.h, grid)
        run(st, dt, int(round(T / dt)))
        ee, _ = I.solitary_wave_1d(x, case.L, 1.0, 0.3, 30.0, case.g, t=st.t)
        errs.append(np.abs(st.eta - ee).max())
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("name,order,run,dts", [
    ("rk4", 4, lambda s, d, k: O.run_rk4(s, d, k, 1e-13), (0.2, 0.1)),
    ("ab2", 2, lambda s, d, k: O.run_ab(s, 2, d, k, 1e-13), (0.04, 0.02)),
    ("ab3", 3, lambda s, d, k: O.run_ab(s, 3, d, k, 1e-13), (0.04, 0.02)),
    ("ab4", 4, lambda s, d, k: O.run_ab(s, 4, d, k, 1e-13), (0.04, 0.02)),
    ("sbdf2", 2, lambda s, d, k: O.run_sbdf2(s, d, k, 1e-13), (0.04, 0.02)),
])
def test_observed_order(name, order, run, dts):
    """Table 1 / Eq:ERK coefficients give the expected convergence order."""
    (p,) = _order_errors(run, dts)
    assert abs(p - order) < 0.35, (name, p)


def test_multistep_tables_consistency():
    for s in (2, 3, 4):
        a, b = O.AB_A[s], O.AB_B[s]
        assert abs(sum(a)) < 1e-15
        assert abs(sum(j * a[j] for j in range(s + 1)) - sum(b)) < 1e-14
    a, b, c = O.SBDF2_A, O.SBDF2_B, O.SBDF2_C
    assert abs(sum(a)) < 1e-15 and abs(sum(j * a[j] for j in range(3)) - sum(b)) < 1e-15
    assert sum(c) == sum(b)      # extrapolation of A p is consistent


def _shelf_state(n=256):
    case = I.shelf_case(n=n, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, w=5.0)
    grid = O.make_grid(1, case.n, case.L, case.g)
    return case, O.init_state(case.eta, case.u, case.h, grid)


def test_mass_conserved_to_roundoff_all_schemes():
    """m = integral zeta is invariant for every scheme (spectral divergence has zero mean)."""
    for run in (lambda s: O.run_rk4(s, 0.05, 4), lambda s: O.run_ab(s, 3, 0.05, 6),
                lambda s: O.run_sbdf2(s, 0.02, 6)):
        case, st = _shelf_state()
        cell = case.L / case.n
        m0 = O.mass(st.eta, st.h, cell)
        run(st)
        assert abs(O.mass(st.eta, st.h, cell) - m0) < 1e-12 * np.abs(st.eta - st.h).sum() * cell


def test_energy_conserved_over_shelf_pins_forcing():
    """E = 1/2 int [g zeta^2 + u.G u] (the flat-bottom energy of the conservation remark
    with the kinetic energy 1/2 B[u,u]) is conserved by the SGN equations with bathymetry;
    RK4's drift vanishes at 4th order.  A wrong term or sign in F, or the other reading of
    (u.grad)^2 h, leaves an O(1e-3) drift."""
    drifts = []
    for dt in (0.04, 0.02):
        case, st = _shelf_state()
        E0 = O.energy(st)
        O.run_rk4(st, dt, int(round(1.2 / dt)), 1e-13)
        drifts.append(abs(O.energy(st) - E0) / E0)
    assert drifts[0] < 2e-6 and drifts[1] < drifts[0] / 10


def test_planted_forcing_mistake_breaks_energy_pin(monkeypatch):
    """The energy pin is sensitive: dropping the eta*m*s term of F leaves a visible drift."""
    def rhs_bad(eta, u, h, hx, L, g):
        d = O.deriv(u, L)
        m = O.deriv(eta * u, L)
        s = hx * u
        S = u * O.deriv(s, L)
        Q = u * O.deriv(d, L) - d * d
        Phi = eta ** 3 * Q / 3 + eta ** 2 * m * d + eta ** 2 * S / 2          # eta m s dropped
        Psi = eta ** 2 * Q / 2 + eta * m * d + eta * S + m * s
        F = O.deriv(Phi, L) - hx * Psi
        return -m, -g * eta * O.deriv(eta - h, L) - O.deriv(eta * u * u, L) + F
    monkeypatch.setattr(O, "rhs_1d", rhs_bad)
    case, st = _shelf_state()
    E0 = O.energy(st)
    O.run_rk4(st, 0.04, 30, 1e-13)
    assert abs(O.energy(st) - E0) / E0 > 1e-5


def _manufactured_error(scheme, order, dt, n=64, t_final=0.5):
    x = np.arange(n) / n
    h, eta, u, _, _ = O.manufactured_1d(x, 0.0)
    st = O.init_state(eta, u, h, O.make_grid(1, n, 1.0, 1.0))
    st.forcing = lambda t: O.manufactured_forcing_1d(x, t, 1.0, 1.0)
    steps = int(round(t_final / dt))
    if scheme == "rk4":
        O.run_rk4(st, dt, steps, 1e-13)
    elif scheme == "ab":
        O.run_ab(st, order, dt, steps, 1e-13)
    else:
        O.run_sbdf2(st, dt, steps, 1e-13)
    _, e1, u1, _, _ = O.manufactured_1d(x, st.t)
    return max(np.abs(st.eta - e1).max(), np.abs(st.u - u1).max())


@pytest.mark.parametrize("scheme,order,dts,min_order", [
    ("rk4", 0, (1 / 50, 1 / 100), 3.8), ("ab", 2, (1 / 200, 1 / 400), 1.9),
    ("ab", 3, (1 / 200, 1 / 400), 2.7), ("ab", 4, (1 / 200, 1 / 400), 3.8),
    ("sbdf2", 0, (1 / 800, 1 / 1600), 1.9)])
def test_forced_schemes_converge_to_manufactured_solution(scheme, order, dts, min_order):
    """Test 1 of §6.4: with the oracle's forcing (S_eta = eta*_t - f_eta, S_U = d/dt(G u*) -
    f_U) every scheme converges to the closed-form (eta*, u*) at its order.  A slip in the
    forcing, in d/dt G, or in a scheme's stage times leaves an O(1) error or drops the
    order."""
    e = [_manufactured_error(scheme, order, dt) for dt in dts]
    assert e[1] < 5e-3
    assert math.log2(e[0] / e[1]) >= min_order, e


def test_manufactured_forcing_fixture_is_the_oracles():
    """tests/golden/manufactured_forcing.json (written by make_manufactured_forcing.py from
    the oracle) is the oracle's forcing: the stored series regenerates exactly and, evaluated
    through the input module's grouping by time function, equals the oracle's forcing at
    times between the fitting samples."""
    import importlib.util
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec_ = importlib.util.spec_from_file_location(
        "make_mf", os.path.join(here, "make_manufactured_forcing.py"))
    mk = importlib.util.module_from_spec(spec_)
    spec_.loader.exec_module(mk)
    stored = json.load(open(os.path.join(here, "manufactured_forcing.json")))
    for part, idx in (("eta", 0), ("U", 1)):
        fresh = mk.series(lambda x, t: O.manufactured_forcing_1d(x, t, 1.0, 1.0, 10.0)[idx])
        assert [e[:4] for e in fresh] == [e[:4] for e in stored[part]]
        scale = max(abs(e[4]) for e in fresh)
        assert max(abs(a[4] - b[4]) for a, b in zip(fresh, stored[part])) <= 1e-13 * scale
    x = I.grid_1d(32, 1.0)
    pe, pu, om, th = I.series_forcing_1d(stored, x)
    for t in (0.03, 0.5, 0.91):
        se, sU = O.manufactured_forcing_1d(x, t, 1.0, 1.0, 10.0)
        w = np.cos(om * t + th)
        assert np.abs(w @ pe - se).max() <= 1e-12 * np.abs(se).max()
        assert np.abs(w @ pu - sU).max() <= 1e-12 * np.abs(sU).max()


def test_2d_plane_wave_matches_1d_evolution():
    """A y-independent 2d solitary wave evolves like the 1d one (§6.5 sanity check)."""
    n, ny, L = 64, 4, 40.0
    case = I.solitary_case(n=n, L=L, a=0.2, x0=20.0, g=9.81)
    g1 = O.make_grid(1, n, L, 9.81)
    s1 = O.init_state(case.eta, case.u, case.h, g1)
    O.run_rk4(s1, 0.02, 5, 1e-13)
    g2 = O.make_grid(2, n, L, 9.81, ny=ny, Ly=5.0)
    E = np.tile(case.eta, (ny, 1))
    U = np.stack([np.tile(case.u, (ny, 1)), np.zeros((ny, n))])
    s2 = O.init_state(E, U, np.ones((ny, n)), g2)
    O.run_rk4(s2, 0.02, 5, 1e-13)
    np.testing.assert_allclose(s2.eta, np.tile(s1.eta, (ny, 1)), atol=1e-11)
    np.testing.assert_allclose(s2.u[0], np.tile(s1.u, (ny, 1)), atol=1e-11)
    assert np.abs(s2.u[1]).max() < 1e-11


def test_sbdf2_zero_stability_region():
    """Eq:ZeroS3 for SBDF2 is bounded iff the eigenvalues of A^{-1}G lie in (0, 4/3)."""
    lam_max = GOLDEN["sbdf2_zero_stability"]["lambda_max_stable"]
    for lam, stable in ((0.05, True), (1.0, True), (1.3, True), (1.36, False), (2.0, False)):
        roots = np.roots([1.0, -2.0 * (1.0 - lam), 1.0 - lam])
        assert (np.abs(roots).max() < 1.0) == stable == (lam < lam_max)
    n = 32
    _, h, eta, _ = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    c = O.precond_coeffs(eta, hx)
    Gd = O.dense_G_1d(eta, hx, 1.0)
    lam_top = O.generalized_eigenvalues(Gd, O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0)).max()
    assert O.sbdf2_zero_stability_growth(Gd, O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0)) < 10
    s = 0.7 * lam_top / lam_max                     # pushes the top eigenvalue past 4/3
    assert O.sbdf2_zero_stability_growth(
        Gd, O.dense_A_1d(s * c["sigma"], s * c["alpha"], n, 1.0), nsteps=400) > 1e3


# ---------------------------------------------------------------------------- GMRES option

def _dense_case(dim):
    if dim == 1:
        n = 16
        _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
        gh = O.deriv(h, 1.0)
        grid = O.make_grid(1, n, 1.0, 1.0)
        c = O.precond_coeffs(eta, gh)
        Gd = O.dense_G_1d(eta, gh, 1.0)
        Ad = O.dense_A_1d(c["sigma"], c["alpha"], n, 1.0)
        return eta, gh, b, grid, c, Gd, Ad, b.shape
    n = 8
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, 1.0, 1.0)
    gh = O.grad(h, (1.0, 1.0))
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    c = O.precond_coeffs(eta, gh)
    Gd = O.dense_G_2d(eta, gh, 1.0, 1.0)
    Ad = O.dense_A_2d(c["sigma"], c["alpha"], n, n, 1.0, 1.0)
    return eta, gh, rhs, grid, c, Gd, Ad, rhs.shape


@pytest.mark.parametrize("dim", [1, 2])
def test_gmres_iterates_minimise_the_residual_over_the_krylov_space(dim):
    """The k-th GMRES iterate from x0 = 0 minimises sqrt(r.A^{-1}r), r = b - G x, over x in
    A^{-1} span{b, M b, ..., M^{k-1} b} with M = G A^{-1}: brute force with the dense
    matrices of Def:MatrixM (no matrix-free operator, no Arnoldi), a Cholesky factor
    A = C C^T, and a least-squares solve of min ||C^{-1}(b - G Z c)||."""
    eta, gh, b, grid, c, Gd, Ad, shape = _dense_case(dim)
    x, steps, _, _, hist = O.gmres(lambda v: O.apply_G(eta, gh, v, grid),
                                   lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid),
                                   b, rtol=1e-14, restart=40, maxit=6, history=True)
    assert steps == 6 and len(hist) == 6
    Ainv = np.linalg.inv(Ad)
    Ci = np.linalg.inv(np.linalg.cholesky(Ad))
    M = Gd @ Ainv
    bf = b.ravel()
    K = [bf]
    for k in range(1, 7):
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        Z = Ainv @ Q
        coef, *_ = np.linalg.lstsq(Ci @ Gd @ Z, Ci @ bf, rcond=None)
        xb = Z @ coef
        assert np.linalg.norm(hist[k - 1].ravel() - xb) <= 1e-9 * np.linalg.norm(xb), k
        K.append(M @ K[-1])
    res = [np.linalg.norm(Ci @ (bf - Gd @ h_.ravel())) for h_ in hist]
    assert all(r1 <= r0 * (1 + 1e-12) for r0, r1 in zip(res, res[1:]))


def test_gmres_reaches_the_lu_solution_within_n_steps():
    """Without restarts GMRES is exact after at most N steps (the Krylov space fills R^N):
    the solution equals a dense LU solve of the Def:MatrixM matrix."""
    eta, gh, b, grid, c, Gd, Ad, _ = _dense_case(1)
    x, steps, ratio, cycles = O.gmres(lambda v: O.apply_G(eta, gh, v, grid),
                                      lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid),
                                      b, rtol=1e-13, restart=16, maxit=16)
    xs = np.linalg.solve(Gd, b)
    assert steps <= 16 and cycles == 1 and ratio <= 1e-13
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_gmres_one_step_when_A_equals_G():
    """Flat bottom and constant depth: G = A exactly (§4), so G A^{-1} = I and GMRES stops
    after one step, with x = A^{-1} b."""
    n, L = 64, 5.0
    eta = np.full(n, 1.3)
    gh = np.zeros(n)
    b = np.cos(2 * np.pi * I.grid_1d(n, L) / L) + 0.3
    grid = O.make_grid(1, n, L, 1.0)
    x, steps, ratio, cycles, c = O.gmres_G(eta, gh, b, grid, rtol=1e-13)
    assert steps == 1 and ratio <= 1e-13
    np.testing.assert_allclose(O.apply_G(eta, gh, x, grid), b, atol=1e-13)


def test_gmres_agrees_with_pcg_and_restarts_cost_steps():
    """On Eq:Testproblem (n = 256) GMRES(30) and PCG reach the same solution of the SPD
    system; GMRES(5) does too, in more steps; every run's true residual is below rtol."""
    n = 256
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    xp, _, _, c = O.solve_G(eta, hx, b, grid, rtol=1e-14, maxit=5000)
    x30, s30, r30, _, _ = O.gmres_G(eta, hx, b, grid, rtol=1e-11, restart=30)
    x5, s5, r5, cyc5, _ = O.gmres_G(eta, hx, b, grid, rtol=1e-11, restart=5, maxit=5000)
    Ainv = lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid)
    for x, r in ((x30, r30), (x5, r5)):
        assert r <= 1e-11
        res = b - O.apply_G(eta, hx, x, grid)
        assert math.sqrt(res @ Ainv(res)) <= 1e-11 * math.sqrt(b @ Ainv(b))
        assert np.linalg.norm(x - xp) <= 1e-11 * math.sqrt(c["kappa_ub"]) * 50 * np.linalg.norm(xp)
    assert s5 > s30 and cyc5 >= s5 // 5
    z, s0, r0, c0, _ = O.gmres_G(eta, hx, np.zeros(n), grid)
    assert s0 == 0 and r0 == 0.0 and c0 == 0 and not z.any()


# ---------------------------------------------------------------------------- dealiasing

@pytest.mark.parametrize("n", [16, 64, 256])
def test_dealias_is_the_two_thirds_projection(n):
    """A projection (P P = P) that keeps every trig mode with |j| <= n/3 exactly and removes
    every mode above it, Nyquist included."""
    x = I.grid_1d(n, 1.0)
    for j in range(0, n // 2 + 1):
        for f in (np.cos(2 * np.pi * j * x), np.sin(2 * np.pi * j * x)):
            if not f.any():
                continue
            keep = j <= n / 3.0
            np.testing.assert_allclose(O.dealias_1d(f), f if keep else 0 * f, atol=1e-13)
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n)
    np.testing.assert_allclose(O.dealias_1d(O.dealias_1d(f)), O.dealias_1d(f), atol=1e-14)


@pytest.mark.parametrize("n", [24, 64, 512])
def test_dealias_removes_quadratic_aliasing(n):
    """For f, g limited to |j| <= K with 3K < n, P(f g) formed on the n-point grid equals the
    exact product (formed on a 2n-point grid, where nothing aliases) truncated to
    |j| <= n/3: the aliased modes of a quadratic product land at |j| >= n - 2K > n/3 and
    the projection removes them.  (n = 24 has 3K < n only up to K = 7.)"""
    rng = np.random.default_rng(7)
    K = (n - 1) // 3

    def band():
        c = np.zeros(n, dtype=complex)
        c[1:K + 1] = rng.standard_normal(K) + 1j * rng.standard_normal(K)
        c[0] = rng.standard_normal()
        c[n - K:] = np.conj(c[1:K + 1][::-1])
        return c

    cf, cg = band(), band()
    f, g = np.real(np.fft.ifft(cf)) * n, np.real(np.fft.ifft(cg)) * n

    def on_2n(c):                                  # the same trig polynomial sampled on 2n points
        C = np.zeros(2 * n, dtype=complex)
        C[:K + 1] = c[:K + 1]
        C[2 * n - K:] = c[n - K:]
        return np.real(np.fft.ifft(C)) * 2 * n

    prod2 = on_2n(cf) * on_2n(cg)
    P2 = np.fft.fft(prod2) / (2 * n)
    Kc = int(n // 3)                               # the projection's cut-off
    exact = np.zeros(n, dtype=complex)
    exact[:Kc + 1] = P2[:Kc + 1]
    exact[n - Kc:] = P2[2 * n - Kc:]
    want = np.real(np.fft.ifft(exact)) * n
    got = O.dealias_1d(f * g)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    assert np.abs(f * g - want).max() > 1e-3 * np.abs(want).max()   # aliasing was there


def test_dealias_2d_is_the_tensor_product_projection():
    """2d: a mode e^{i(jx x + jy y)} survives iff |jx| <= nx/3 and |jy| <= ny/3; the
    projection of a product field factorises into the 1d projections."""
    nx, ny = 32, 16
    X, Y = I.grid_2d(nx, ny, 1.0, 1.0)
    for jx in (0, 5, 10, 11, 16):
        for jy in (0, 3, 5, 6, 8):
            f = np.cos(2 * np.pi * (jx * X + jy * Y))
            keep = jx <= nx / 3.0 and jy <= ny / 3.0
            np.testing.assert_allclose(O.dealias_2d(f), f if keep else 0 * f, atol=1e-13)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(nx), rng.standard_normal(ny)
    np.testing.assert_allclose(O.dealias_2d(b[:, None] * a[None, :]),
                               O.dealias_1d(b)[:, None] * O.dealias_1d(a)[None, :], atol=1e-13)


# ---------------------------------------------------------------------------- non-constraint form

def test_dGdt_matches_a_finite_difference_in_eta():
    """d/dt (G_eta u) with u fixed is the eta-derivative of Def:G in the direction eta_t:
    against a central difference of the matrix-free operator (no shared formula)."""
    n, L = 128, 10.0
    x = I.grid_1d(n, L)
    h = 1.0 + 0.3 * np.sin(2 * np.pi * x / L)
    hx = O.deriv(h, L)
    eta = h + 0.2 * np.cos(2 * np.pi * x / L) ** 2
    u = np.sin(4 * np.pi * x / L) + 0.3
    e = np.cos(6 * np.pi * x / L)
    eps = 1e-5
    fd = (O.apply_G_1d(eta + eps * e, hx, u, L) - O.apply_G_1d(eta - eps * e, hx, u, L)) / (2 * eps)
    an = O.dGdt_1d(eta, e, hx, u, np.zeros(n), L)
    assert np.abs(fd - an).max() <= 1e-8 * np.abs(an).max()


@pytest.mark.parametrize("n", [64, 256])
def test_momentum_form_equals_the_constraint_form(n):
    """Eq:MomEq (u_t-free terms M) and the DAE form must agree: G u_t = M and
    d/dt(G u) = f_U give M = f_U - (d/dt G) u with eta_t = f_eta.  Two transcriptions (Eq:MomEq
    against Def:bigF with the product rule) agree to the spectral accuracy of the grid."""
    L = 20.0
    x = I.grid_1d(n, L)
    th = 2 * np.pi * x / L                         # smooth periodic fields (entire functions)
    h = 1.0 - 0.3 * np.exp(np.cos(th) - 1.0)
    hx = O.deriv(h, L)
    eta = h + 0.15 * np.exp(np.cos(th + 1.0) - 1.0)
    u = 0.3 * np.sin(th) * np.exp(0.5 * np.cos(2 * th))
    fe, fU = O.rhs_1d(eta, u, h, hx, L, 9.81)
    fe2, M = O.rhs_nc_1d(eta, u, h, hx, L, 9.81)
    np.testing.assert_allclose(fe2, fe, atol=1e-14)
    other = fU - O.dGdt_1d(eta, fe, hx, u, np.zeros(n), L)
    err = np.abs(M - other).max() / np.abs(M).max()
    assert err <= 1e-12, err


def test_nonconstraint_rk4_solitary_wave_and_constraint_form():
    """Flat bottom: the non-constraint RK4 follows the exact translate (§6) as the
    constraint-form RK4 does, and the two discretisations differ at fourth order in dt."""
    c = I.solitary_case(n=256, L=100.0, a=0.2, x0=25.0, g=9.81)
    grid = O.make_grid(1, c.n, c.L, c.g)
    x = I.grid_1d(c.n, c.L)
    diffs = []
    for dt, k in ((0.04, 10), (0.02, 20)):
        a = O.init_state(c.eta, c.u, c.h, grid)
        b = O.init_state(c.eta, c.u, c.h, grid)
        O.run_rk4_nc(a, dt, k, 1e-13)
        O.run_rk4(b, dt, k, 1e-13)
        ee, _ = I.solitary_wave_1d(x, c.L, 1.0, 0.2, 25.0, c.g, t=0.4)
        assert np.abs(a.eta - ee).max() < 1e-6
        assert np.abs(O.apply_G_1d(a.eta, a.gradh, a.u, c.L) - a.U).max() < 1e-12
        diffs.append(np.abs(a.eta - b.eta).max())
    assert math.log2(diffs[0] / diffs[1]) > 3.5, diffs


def test_momentum_form_equals_the_constraint_form_2d():
    """The 2d Eq:MomEq terms against the 2d DAE form with the product rule (dG/dt in 2d,
    itself checked against a central difference of the operator in eta)."""
    nx, ny, Lx, Ly = 48, 32, 20.0, 12.0
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    ax, ay = 2 * np.pi * X / Lx, 2 * np.pi * Y / Ly
    h = 1.0 - 0.3 * np.exp(np.cos(ax) + np.cos(ay) - 2.0)
    gh = O.grad(h, (Lx, Ly))
    eta = h + 0.15 * np.exp(np.cos(ax + 1.0) * np.cos(ay) - 1.0)
    u = np.stack([0.3 * np.sin(ax) * np.exp(0.5 * np.cos(ay)),
                  0.2 * np.cos(ay + 0.5) * np.exp(0.3 * np.sin(ax))])
    e = np.cos(ax) * np.sin(2 * ay)
    eps = 1e-5
    fd = (O.apply_G_2d(eta + eps * e, gh, u, Lx, Ly) -
          O.apply_G_2d(eta - eps * e, gh, u, Lx, Ly)) / (2 * eps)
    an = O.dGdt_2d(eta, e, gh, u, Lx, Ly)
    assert np.abs(fd - an).max() <= 1e-8 * np.abs(an).max()
    fe, fU = O.rhs_2d(eta, u, h, gh, Lx, Ly, 9.81)
    fe2, M = O.rhs_nc_2d(eta, u, h, gh, Lx, Ly, 9.81)
    np.testing.assert_allclose(fe2, fe, atol=1e-14)
    other = fU - O.dGdt_2d(eta, fe, gh, u, Lx, Ly)
    assert np.abs(M - other).max() <= 1e-12 * np.abs(M).max()
