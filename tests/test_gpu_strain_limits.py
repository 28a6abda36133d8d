"""GPU parity of strain limits (singular values of each triangle's deformation gradient
clamped to [s_min, s_max]): the step against the oracle's limited step, in both forms and
both execution modes, on deformed cells whose triangles fall below, inside and above the
limits; the argument checks; the adjoints refuse limited types."""
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


def test_strain_limit_arguments_and_adjoints():
    nat = _native()
    m = I.rbc_mesh(1)
    base = I.RBC_MATERIAL.as_tuple() + (0.0, 0.0)
    for bad in ((1.1, 1.2), (0.8, 0.9), (-0.1, 1.1), (0.9, float("inf")), (float("nan"), 1.1), (0.0, 1.1)):
        with pytest.raises(nat.NpfemError, match="strain limits"):
            nat.CellType(m.verts, m.tris, base + bad, 0.1)
    b = I.single_rbc(subdiv=1)
    t = nat.CellType(m.verts, m.tris, base + (0.9, 1.1), b.dt)
    batch = nat.Batch([t], [0], nat.FP64)
    dev = torch.device("cuda:0")
    X = torch.tensor(b.x, device=dev)
    g = [torch.zeros_like(X) for _ in range(5)]
    gw = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    with pytest.raises(nat.NpfemError, match="strain limits"):
        batch.step_adjoint(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw, iters_default=3)
    with pytest.raises(nat.NpfemError, match="strain limits"):
        batch.step_adjoint_implicit(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw)
