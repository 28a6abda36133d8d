"""GPU parity of Rayleigh damping (materials with c_alpha, c_beta): the step against the
oracle's damped step, in both forms and both execution modes, plus the argument checks
(negative or non-finite damping rejected)."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
FP32_BAR = 1e-5
# (c_alpha 1/us, c_beta us) per cell type of the batch
DAMPING = [(0.5, 1.0), (2.0, 0.0), (0.0, 3.0)]


def _native():
    from paper_2011_04332_b300 import native
    return native


def _materials(b):
    return [t.material.as_tuple() + DAMPING[k % len(DAMPING)] for k, t in enumerate(b.types)]


def _run(b, prec, split=True, steps=2):
    nat = _native()
    mats = _materials(b)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    batch = nat.Batch(types, b.type_of_cell, prec)
    batch.set_mode(split)
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, mats[k], b.dt) for k, t in enumerate(b.types)]
    dev = torch.device("cuda:0")
    tdt = torch.float64 if prec == nat.FP64 else torch.float32
    x, v, f = b.x.copy(), b.v.copy(), b.f.copy()
    if prec == nat.FP32FORM:
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    bar = FP64_BAR if prec == nat.FP64 else FP32_BAR
    for s in range(steps):
        X, V, F = (torch.tensor(a, dtype=tdt, device=dev) for a in (x, v, f))
        it = torch.tensor(b.iters, device=dev)
        st = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
        al = torch.zeros((b.ncells, 8), dtype=torch.float64, device=dev)
        batch.step(X, V, F, iters=it, status=st, alpha_log=al)
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
            if prec == nat.FP64:
                k = min(int(b.iters[c]), 8)
                assert np.array_equal(al[c, :k].cpu().numpy(), np.array(ref["alphas"][c][:k])), (s, c)
        x, v = ref["x"], ref["v"]
        if prec == nat.FP32FORM:
            x, v = (a.astype(np.float32).astype(np.float64) for a in (x, v))
    return batch


@pytest.mark.parametrize("mode", ["split", "fused"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_damped_small_mixed_batch(mode, prec):
    """Three small types with different damping (mass only, stiffness only, both),
    ragged iteration counts, non-zero velocities; two consecutive steps."""
    nat = _native()
    _run(I.small_mixed_batch(), nat.FP64 if prec == "fp64" else nat.FP32FORM, split=(mode == "split"))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_damped_placed_rbcs(prec):
    """24 placed 642-vertex RBCs with c_alpha = 0.5 /us, c_beta = 1 us."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=24, seed=1001, velocity_sigma=0.02)
    _run(b, nat.FP64 if prec == "fp64" else nat.FP32FORM)


def test_damping_arguments():
    nat = _native()
    m = I.rbc_mesh(1)
    for bad in ((-0.1, 0.0), (0.0, -1.0), (float("nan"), 0.0), (0.0, float("inf"))):
        with pytest.raises(nat.NpfemError, match="damping"):
            nat.CellType(m.verts, m.tris, I.RBC_MATERIAL.as_tuple() + bad, 0.1)
