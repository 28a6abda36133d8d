"""GPU implicit-function adjoint (gradients through the converged step): against the
oracle's implicit adjoint, against finite differences of the converged GPU step itself,
the CG status bit, and argument errors."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITERS, TOL = 300, 1e-12     # forward: run to convergence (fused kernel, no iteration bound)


def _native():
    from paper_2011_04332_b300 import native
    return native


def _materials(b, damping):
    return [t.material.as_tuple() + tuple(damping) for t in b.types]


def _batch(b, damping=()):
    nat = _native()
    mats = _materials(b, damping)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    batch = nat.Batch(types, b.type_of_cell, nat.FP64)
    batch.set_mode(False)
    return types, batch


def _adjoint(batch, b, gxn, gvn, cg_tol=1e-13, cg_max=500):
    dev = torch.device("cuda:0")
    X, V, F = (torch.tensor(a, device=dev) for a in (b.x, b.v, b.f))
    GXN, GVN = torch.tensor(gxn, device=dev), torch.tensor(gvn, device=dev)
    gx, gv, gf = (torch.zeros_like(X) for _ in range(3))
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
    it = torch.full((b.ncells,), ITERS, dtype=torch.int32, device=dev)
    batch.step_adjoint_implicit(X, V, F, GXN, GVN, gx, gv, gf, gw, iters=it, tol=TOL, cg_tol=cg_tol,
                                cg_max_iters=cg_max, status=st)
    torch.cuda.synchronize()
    return (gx.cpu().numpy(), gv.cpu().numpy(), gf.cpu().numpy(), gw.cpu().numpy(), st.cpu().numpy())


def _forward(batch, b, x, v, f):
    dev = torch.device("cuda:0")
    X, V, F = (torch.tensor(a, device=dev) for a in (x, v, f))
    it = torch.full((b.ncells,), ITERS, dtype=torch.int32, device=dev)
    res = torch.zeros(b.ncells, dtype=torch.float64, device=dev)
    batch.step(X, V, F, iters=it, residual=res, tol=TOL)
    torch.cuda.synchronize()
    return X.cpu().numpy(), V.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("damping", [(), (0.5, 1.0)])
def test_implicit_adjoint_matches_oracle(damping):
    """Small mixed batch (42-vertex RBC and platelet, 162-vertex RBC), without and with
    Rayleigh damping: every gradient against the oracle's implicit adjoint at its own
    converged state."""
    b = I.small_mixed_batch()
    _, batch = _batch(b, damping)
    mats = _materials(b, damping)
    rng = np.random.default_rng(51)
    gxn = rng.standard_normal(b.x.shape)
    gvn = 0.1 * rng.standard_normal(b.x.shape)
    gx, gv, gf, gw, st = _adjoint(batch, b, gxn, gvn)
    assert np.all(st == 0), st
    for c in range(b.ncells):
        s = b.cell_slice(c)
        t = b.types[int(b.type_of_cell[c])]
        ct = O.CellType(t.mesh.verts, t.mesh.tris, mats[int(b.type_of_cell[c])], b.dt)
        xc, vc, fc = b.cell_state(c)
        r = O.step(ct.rest, ct.solver, xc, vc, fc, 400, tol=1e-13)
        assert r.residual < 1e-11
        rx, rv, rf, rw = O.implicit_adjoint(ct, xc, vc, fc, r.x, gxn[:, s].T, gvn[:, s].T)
        for got, ref in ((gx[:, s].T, rx), (gv[:, s].T, rv), (gf[:, s].T, rf)):
            assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref)), c
        assert np.allclose(gw[c], rw, rtol=1e-7, atol=1e-9 * np.max(np.abs(rw))), (c, gw[c], rw)


def test_implicit_adjoint_matches_gpu_finite_differences():
    """L = gx . x* + gv . v* with x* from the converged GPU step: central differences of
    L in a few position, velocity and force components against the implicit gradients."""
    b = I.homogeneous_rbc_batch(ncells=4, seed=1001, velocity_sigma=0.02)
    _, batch = _batch(b)
    rng = np.random.default_rng(53)
    gxn = rng.standard_normal(b.x.shape)
    gvn = 0.1 * rng.standard_normal(b.x.shape)
    gx, gv, gf, gw, st = _adjoint(batch, b, gxn, gvn)
    assert np.all(st == 0)

    def loss(x, v, f):
        xs, vs, res = _forward(batch, b, x, v, f)
        assert np.all(res < 1e-10)
        return float(np.sum(gxn * xs) + np.sum(gvn * vs))

    for arr_name, grad, h in (("x", gx, 1e-4), ("v", gv, 1e-3), ("f", gf, 1e-4)):
        for k in rng.integers(0, b.n_total, 3):
            d = int(rng.integers(0, 3))
            arrs = {"x": b.x.copy(), "v": b.v.copy(), "f": b.f.copy()}
            base = arrs[arr_name][d, k]
            arrs[arr_name][d, k] = base + h
            lp = loss(arrs["x"], arrs["v"], arrs["f"])
            arrs[arr_name][d, k] = base - h
            lm = loss(arrs["x"], arrs["v"], arrs["f"])
            fd = (lp - lm) / (2 * h)
            assert grad[d, k] == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.max(np.abs(grad))), (arr_name, d, k)


def test_cg_budget_sets_status_bit():
    nat = _native()
    b = I.small_mixed_batch()
    _, batch = _batch(b)
    rng = np.random.default_rng(55)
    gx, gv, gf, gw, st = _adjoint(batch, b, rng.standard_normal(b.x.shape), np.zeros_like(b.x), cg_max=1)
    assert np.all((st & 16) == 16), st
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gw))


def test_implicit_adjoint_arguments():
    nat = _native()
    b = I.single_rbc(subdiv=1)
    dev = torch.device("cuda:0")
    X = torch.tensor(b.x, device=dev)
    g = [torch.zeros_like(X) for _ in range(5)]
    gw = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    t = nat.CellType(b.types[0].mesh.verts, b.types[0].mesh.tris, b.types[0].material.as_tuple(), b.dt)
    batch = nat.Batch([t], [0], nat.FP64)
    for kw in ({"cg_tol": 0.0}, {"cg_tol": float("nan")}, {"cg_max_iters": 0}):
        with pytest.raises(nat.NpfemError, match="cg_"):
            batch.step_adjoint_implicit(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw, **kw)
    batch.set_collisions(0.5, 0.05, 10.0)
    with pytest.raises(nat.NpfemError, match="collisions"):
        batch.step_adjoint_implicit(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw)
    b32 = nat.Batch([t], [0], nat.FP32FORM)
    with pytest.raises(nat.NpfemError, match="FP64"):
        b32.step_adjoint_implicit(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw)
