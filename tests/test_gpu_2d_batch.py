"""2d batches: several 2d instances on one grid in one layout, solved together (the mixed
solve's float32 inner PCG of every instance runs in one persistent launch per refinement
pass), against the oracle and against each instance solved alone.

Batch packing: a scalar field holds instance b at [b P, b P + P); a vector field holds the
x components of all instances, then the y components.
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
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64).ravel(), device="cuda")


def pack_scalar(fs):
    return np.concatenate([f.ravel() for f in fs])


def pack_vector(vs):
    return np.concatenate([v[0].ravel() for v in vs] + [v[1].ravel() for v in vs])


def unpack_vector(a, B, ny, nx):
    a = np.asarray(a).reshape(2, B, ny, nx)
    return [a[:, b] for b in range(B)]


def instance(nx, ny, Lx, Ly, seed):
    """Depth over a Gaussian bump (height, radius and centre drawn from the seed), a wave on
    it, and b = G u* for a smooth u* from the oracle's operator."""
    rng = np.random.default_rng(seed)
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    h = I.gaussian_bump_2d(X, Y, Lx, Ly, rng.uniform(0.1, 0.6), rng.uniform(1.0, 5.0) * Lx / 80,
                           rng.uniform(0.3, 0.7) * Lx, rng.uniform(0.3, 0.7) * Ly)
    eta = h + rng.uniform(0.05, 0.3) * np.exp(np.cos(2 * np.pi * X / Lx - rng.uniform(0, 6)) - 1)
    gh = O.grad(h, (Lx, Ly))
    k = int(rng.integers(1, 4))
    us = np.stack([0.3 * np.sin(2 * np.pi * k * X / Lx) * np.cos(4 * np.pi * Y / Ly),
                   0.2 * np.cos(2 * np.pi * X / Lx) + 0.1 * np.sin(2 * np.pi * k * Y / Ly)])
    grid = O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly)
    b = O.apply_G(eta, gh, us, grid)
    return h, eta, gh, b, us, grid


@pytest.mark.parametrize("nx,ny,B", [(32, 16, 3), (64, 64, 5)])
def test_batch_operators_match_oracle(S, nx, ny, B):
    """Gradient, coefficients, operator and A^{-1} on a batch equal the oracle per instance."""
    sgn, ctx = S
    Lx, Ly = 20.0, 10.0
    inst = [instance(nx, ny, Lx, Ly, 100 + i) for i in range(B)]
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)] * B)
    assert lay.points == B * nx * ny
    gh = torch.zeros(2 * B * nx * ny, dtype=torch.float64, device="cuda")
    sgn.spectral_grad(lay, dev(pack_scalar([c[0] for c in inst])), gh)
    for b, v in enumerate(unpack_vector(gh.cpu().numpy(), B, ny, nx)):
        assert rel(v, inst[b][2]) < 1e-12
    eta, ghp = dev(pack_scalar([c[1] for c in inst])), dev(pack_vector([c[2] for c in inst]))
    P = sgn.precond_coeffs(lay, eta, ghp)
    for b in range(B):
        ref = O.precond_coeffs(inst[b][1], inst[b][2])
        assert abs(P[b]["sigma"] - ref["sigma"]) <= 1e-13 * ref["sigma"]
        assert abs(P[b]["alpha"] - ref["alpha"]) <= 1e-13 * ref["alpha"]
    u = dev(pack_vector([c[4] for c in inst]))
    Gu = torch.zeros_like(u)
    sgn.apply_operator(lay, eta, ghp, u, Gu)
    for b, v in enumerate(unpack_vector(Gu.cpu().numpy(), B, ny, nx)):
        assert rel(v, inst[b][3]) < 1e-12
    z = torch.zeros_like(u)
    sgn.precond_solve(lay, P, u, z)
    for b, v in enumerate(unpack_vector(z.cpu().numpy(), B, ny, nx)):
        ref = O.apply_Ainv(inst[b][4], P[b]["sigma"], P[b]["alpha"], inst[b][5])
        assert rel(v, ref) < 1e-12


@pytest.mark.parametrize("nx,ny,B", [(16, 8, 2), (64, 32, 4), (128, 128, 6)])
def test_batch_pcg_matches_oracle_and_alone(S, nx, ny, B):
    """Mixed and float64 batched solves: every instance reaches the known u* and equals the
    same instance solved alone (float64 bitwise: the same single-instance solve)."""
    sgn, ctx = S
    Lx, Ly = 40.0, 20.0
    inst = [instance(nx, ny, Lx, Ly, 7 * i + nx) for i in range(B)]
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)] * B)
    one = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    eta, ghp = dev(pack_scalar([c[1] for c in inst])), dev(pack_vector([c[2] for c in inst]))
    b = dev(pack_vector([c[3] for c in inst]))
    for prec, rtol in ((sgn.PREC_MIXED, 1e-11), (sgn.PREC_FP64, 1e-12)):
        x = torch.zeros_like(b)
        info = sgn.pcg(lay, eta, ghp, b, x, rtol=rtol, maxit=4000, prec=prec)
        xs = unpack_vector(x.cpu().numpy(), B, ny, nx)
        for i in range(B):
            assert info[i]["status"] == 0 and info[i]["ratio"] <= rtol
            assert rel(xs[i], inst[i][4]) < 1e-8
            x1 = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
            i1 = sgn.pcg(one, dev(inst[i][1]), dev(inst[i][2]), dev(inst[i][3]), x1, rtol=rtol,
                         maxit=4000, prec=prec)[0]
            if prec == sgn.PREC_FP64:
                assert np.array_equal(x1.cpu().numpy().reshape(2, ny, nx), xs[i])
                assert i1["iters"] == info[i]["iters"]
            else:
                assert rel(xs[i], x1.cpu().numpy().reshape(2, ny, nx)) < 1e-9
    # small grids: the oracle's own solve
    if nx * ny <= 64 * 32:
        x = torch.zeros_like(b)
        sgn.pcg(lay, eta, ghp, b, x, rtol=1e-12, maxit=4000, prec=sgn.PREC_MIXED)
        for i, v in enumerate(unpack_vector(x.cpu().numpy(), B, ny, nx)):
            ref = O.solve_G(inst[i][1], inst[i][2], inst[i][3], inst[i][5], rtol=1e-14,
                            maxit=4000)[0]
            assert rel(v, ref) < 1e-9


def test_batch_pcg_mixed_outcomes(S):
    """Instances of one batch finish on their own terms: a zero right-hand side (x = 0, no
    iteration), a non-positive depth (reported), and ordinary instances (solved)."""
    sgn, ctx = S
    nx = ny = 32
    B = 4
    inst = [instance(nx, ny, 10.0, 10.0, 50 + i) for i in range(B)]
    etas = [c[1].copy() for c in inst]
    etas[2][4, 4] = -0.3
    bs = [c[3] for c in inst]
    bs[1] = np.zeros_like(bs[1])
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 10.0, ny=ny, Ly=10.0, g=9.81)] * B)
    x = dev(np.ones(2 * B * nx * ny))
    info = sgn.pcg(lay, dev(pack_scalar(etas)), dev(pack_vector([c[2] for c in inst])),
                   dev(pack_vector(bs)), x, rtol=1e-11, maxit=4000, prec=sgn.PREC_MIXED,
                   check=False)
    xs = unpack_vector(x.cpu().numpy(), B, ny, nx)
    assert [i["status"] for i in info] == [0, 0, 7, 0]
    assert info[1]["iters"] == 0 and np.all(xs[1] == 0.0)
    for i in (0, 3):
        assert rel(xs[i], inst[i][4]) < 1e-8


def test_batch_rejections(S):
    sgn, ctx = S
    g = sgn.Grid(2, 16, 1.0, ny=16, Ly=1.0)
    with pytest.raises(sgn.SgnError):
        sgn.Layout(ctx, [g, sgn.Grid(2, 32, 1.0, ny=16, Ly=1.0)])
    with pytest.raises(sgn.SgnError):
        sgn.Layout(ctx, [g] * 33)
    lay = sgn.Layout(ctx, [g] * 2)
    z = torch.zeros(2 * 2 * 256, dtype=torch.float64, device="cuda")
    zs = torch.zeros(2 * 256, dtype=torch.float64, device="cuda") + 1.0
    with pytest.raises(sgn.SgnError):
        sgn.rhs(lay, zs, z, zs, z, zs.clone(), z.clone())
    with pytest.raises(sgn.SgnError):
        sgn.State(lay, zs, z, z.clone(), zs.clone(), z.clone())
    with pytest.raises(sgn.SgnError):
        sgn.gmres(lay, zs, z, z.clone(), z.clone())


def test_batch_512_mixed_solves(S):
    """Eight 512^2 instances of the bump workload in one batch: each reaches its known u*."""
    sgn, ctx = S
    n, B, L = 512, 8, 80.0
    inst = [instance(n, n, L, L, 900 + i) for i in range(B)]
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, L, ny=n, Ly=L, g=9.81)] * B)
    eta, ghp = dev(pack_scalar([c[1] for c in inst])), dev(pack_vector([c[2] for c in inst]))
    b = dev(pack_vector([c[3] for c in inst]))
    x = torch.zeros_like(b)
    info = sgn.pcg(lay, eta, ghp, b, x, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    for i, v in enumerate(unpack_vector(x.cpu().numpy(), B, n, n)):
        assert info[i]["status"] == 0 and info[i]["ratio"] <= 1e-10
        assert rel(v, inst[i][4]) < 1e-7
