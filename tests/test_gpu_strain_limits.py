"""GPU parity of strain limits (singular values of each triangle's deformation gradient
clamped to [s_min, s_max]): the step against the oracle's limited step, in both forms and
both execution modes, on deformed cells whose triangles fall below, inside and above the
limits; the argument checks; both adjoints through the clamped projection (the unrolled
adjoint against the oracle's complex-step derivative, the implicit adjoint against the
oracle's implicit adjoint)."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
FP32_BAR = 1e-5
LIMITS = [(0.97, 1.03), (0.9, 1.0), (1.0, 1.05)]     # per cell type of the batch


def _native():
    from paper_2011_04332_b300 import native
    return native


def _materials(b):
    return [t.material.as_tuple() + (0.0, 0.0) + LIMITS[k % len(LIMITS)] for k, t in enumerate(b.types)]


def _deformed(b, seed):
    """Each cell stretched along x by 8 % and squeezed along y by 5 % about its centroid,
    plus small noise: strains on both sides of every type's limits."""
    rng = np.random.default_rng(seed)
    x = b.x.copy()
    for c in range(b.ncells):
        sl = b.cell_slice(c)
        ctr = x[:, sl].mean(axis=1, keepdims=True)
        x[:, sl] = ctr + np.array([[1.08], [0.95], [1.0]]) * (x[:, sl] - ctr)
    return x + 0.005 * rng.standard_normal(x.shape)


def _run(b, prec, split=True, steps=2):
    nat = _native()
    mats = _materials(b)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    batch = nat.Batch(types, b.type_of_cell, prec)
    batch.set_mode(split)
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    dev = torch.device("cuda:0")
    tdt = torch.float64 if prec == nat.FP64 else torch.float32
    x, v, f = _deformed(b, 71), b.v.copy(), b.f.copy()
    if prec == nat.FP32FORM:
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    bar = FP64_BAR if prec == nat.FP64 else FP32_BAR
    for s in range(steps):
        X, V, F = (torch.tensor(a, dtype=tdt, device=dev) for a in (x, v, f))
        it = torch.tensor(b.iters, device=dev)
        st = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
        batch.step(X, V, F, iters=it, status=st)
        torch.cuda.synchronize()
        ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, b.iters)
        xg, vg = X.double().cpu().numpy(), V.double().cpu().numpy()
        for c in range(b.ncells):
            sl = b.cell_slice(c)
            xr = ref["x"][:, sl]
            rad = np.max(np.linalg.norm(xr - xr.mean(axis=1, keepdims=True), axis=0))
            assert np.max(np.abs(xg[:, sl] - xr)) / rad <= bar, (s, c)
            assert np.max(np.abs(vg[:, sl] - ref["v"][:, sl])) * b.dt / rad <= bar, (s, c)
            assert int(st[c]) == ref["status"][c]
        x, v = ref["x"], ref["v"]
        if prec == nat.FP32FORM:
            x, v = (a.astype(np.float32).astype(np.float64) for a in (x, v))


@pytest.mark.parametrize("mode", ["split", "fused"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_limited_small_mixed_batch(mode, prec):
    nat = _native()
    _run(I.small_mixed_batch(), nat.FP64 if prec == "fp64" else nat.FP32FORM, split=(mode == "split"))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_limited_placed_rbcs(prec):
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=12, seed=1001, velocity_sigma=0.02)
    _run(b, nat.FP64 if prec == "fp64" else nat.FP32FORM)


def test_strain_limit_arguments():
    nat = _native()
    m = I.rbc_mesh(1)
    base = I.RBC_MATERIAL.as_tuple() + (0.0, 0.0)
    for bad in ((1.1, 1.2), (0.8, 0.9), (-0.1, 1.1), (0.9, float("inf")), (float("nan"), 1.1), (0.0, 1.1)):
        with pytest.raises(nat.NpfemError, match="strain limits"):
            nat.CellType(m.verts, m.tris, base + bad, 0.1)


def _limited_batch(b):
    nat = _native()
    mats = _materials(b)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    return mats, types, nat.Batch(types, b.type_of_cell, nat.FP64)


def test_unrolled_adjoint_through_strain_limits_against_oracle_forward_mode():
    """Dot-product identity lambda^T (J delta) = (J^T lambda)^T delta between the GPU
    reverse mode and the oracle's complex-step derivative of its limited step, from a
    deformed state whose triangles lie below, inside and above each type's limits; every
    input block separately as well (positions, velocities, forces, weights)."""
    b = I.small_mixed_batch(seed=9, iters=(3, 6))
    mats, types, batch = _limited_batch(b)
    x = _deformed(b, 72)
    rng = np.random.default_rng(9)
    lam_x = rng.standard_normal(b.x.shape)
    lam_v = rng.standard_normal(b.x.shape) * 1e-2
    dx = rng.standard_normal(b.x.shape) * 1e-2
    dv = rng.standard_normal(b.x.shape) * 1e-2
    df = rng.standard_normal(b.x.shape) * 1e-3
    dws = rng.standard_normal((len(b.types), 4))
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    gx, gv, gf = (torch.zeros((3, b.n_total), dtype=torch.float64, device=dev) for _ in range(3))
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
    batch.step_adjoint(T(x), T(b.v), T(b.f), T(lam_x), T(lam_v), gx, gv, gf, gw,
                       iters=torch.tensor(b.iters, device=dev), status=st)
    torch.cuda.synchronize()
    assert int(st.max()) == 0 and int(st.min()) == 0
    gx, gv, gf, gw = (a.cpu().numpy() for a in (gx, gv, gf, gw))

    def jvp(ddx, ddv, ddf, ddw):
        ox, ov = np.zeros_like(b.x), np.zeros_like(b.x)
        for c in range(b.ncells):
            t = int(b.type_of_cell[c])
            ws = np.ones(4, complex) + 1j * 1e-30 * ddw[t]
            ct = O.CellType(b.types[t].mesh.verts, b.types[t].mesh.tris, mats[t], b.dt, ws)
            sl = b.cell_slice(c)
            r = O.step(ct.rest, ct.solver, x[:, sl].T + 1j * 1e-30 * ddx[:, sl].T,
                       b.v[:, sl].T + 1j * 1e-30 * ddv[:, sl].T, b.f[:, sl].T + 1j * 1e-30 * ddf[:, sl].T,
                       int(b.iters[c]), ws)
            ox[:, sl] = (np.imag(r.x) / 1e-30).T
            ov[:, sl] = (np.imag(r.v) / 1e-30).T
        return ox, ov

    def rhs_of(ddx, ddv, ddf, ddw):
        r = np.sum(gx * ddx) + np.sum(gv * ddv) + np.sum(gf * ddf)
        for c in range(b.ncells):
            t = int(b.type_of_cell[c])
            r += np.sum(gw[c] * np.array(mats[t][:4]) * ddw[t])
        return r

    jx, jv = jvp(dx, dv, df, dws)
    lhs = np.sum(lam_x * jx) + np.sum(lam_v * jv)
    assert rhs_of(dx, dv, df, dws) == pytest.approx(lhs, rel=1e-9)
    for blk in range(4):
        d = [np.zeros_like(dx), np.zeros_like(dv), np.zeros_like(df), np.zeros_like(dws)]
        d[blk] = [dx, dv, df, dws][blk]
        jx, jv = jvp(*d)
        l2 = np.sum(lam_x * jx) + np.sum(lam_v * jv)
        assert rhs_of(*d) == pytest.approx(l2, rel=1e-8, abs=1e-12 * abs(lhs)), f"block {blk}"


def test_implicit_adjoint_through_strain_limits_against_oracle():
    """Gradients through the converged limited step against the oracle's implicit adjoint
    (its exact Hessian by complex step through the clamped projection), at 1e-7."""
    b = I.small_mixed_batch(seed=10)
    mats, types, batch = _limited_batch(b)
    batch.set_mode(False)
    x = _deformed(b, 73)
    rng = np.random.default_rng(10)
    gxn = rng.standard_normal(b.x.shape)
    gvn = 0.1 * rng.standard_normal(b.x.shape)
    dev = torch.device("cuda:0")
    X, V, F = (torch.tensor(a, device=dev) for a in (x, b.v, b.f))
    gx, gv, gf = (torch.zeros_like(X) for _ in range(3))
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
    it = torch.full((b.ncells,), 300, dtype=torch.int32, device=dev)
    batch.step_adjoint_implicit(X, V, F, torch.tensor(gxn, device=dev), torch.tensor(gvn, device=dev),
                                gx, gv, gf, gw, iters=it, tol=1e-12, cg_tol=1e-13, cg_max_iters=500, status=st)
    torch.cuda.synchronize()
    assert int(st.max()) == 0, st
    gx, gv, gf, gw = (a.cpu().numpy() for a in (gx, gv, gf, gw))
    for c in range(b.ncells):
        s = b.cell_slice(c)
        t = int(b.type_of_cell[c])
        ct = O.CellType(b.types[t].mesh.verts, b.types[t].mesh.tris, mats[t], b.dt)
        xc, vc, fc = x[:, s].T.copy(), b.v[:, s].T.copy(), b.f[:, s].T.copy()
        r = O.step(ct.rest, ct.solver, xc, vc, fc, 400, tol=1e-13)
        assert r.residual < 1e-11
        rx, rv, rf, rw = O.implicit_adjoint(ct, xc, vc, fc, r.x, gxn[:, s].T, gvn[:, s].T)
        for got, ref in ((gx[:, s].T, rx), (gv[:, s].T, rv), (gf[:, s].T, rf)):
            assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref)), c
        assert np.allclose(gw[c], rw, rtol=1e-7, atol=1e-9 * np.max(np.abs(rw))), (c, gw[c], rw)
