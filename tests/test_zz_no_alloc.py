"""The allocation-free step (npfem_step_noalloc) against the regular batched step.

npfem_step_noalloc exists for callers that are not allowed to allocate device memory
(a host framework whose pool owns all device memory, code running during stream
capture, tools with a device-memory budget fixed at start-up).  It runs the same
step with its workspace in a static device array instead of a batch's workspace.
These tests call it through the C ABI twice in a row and compare each result with
npfem_step on the same inputs, with the parity bars of the oracle tests.  This file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {"fp64": 1e-10, "fp32": 1e-5}


def _rel_err(b, x, xref, radius_from=None):
    """max over cells of |x - xref|_inf / cell radius (of radius_from, default xref)."""
    rf = xref if radius_from is None else radius_from
    worst = 0.0
    for c in range(b.ncells):
        s = b.cell_slice(c)
        xr = rf[:, s]
        rad = np.max(np.linalg.norm(xr - xr.mean(axis=1, keepdims=True), axis=0))
        worst = max(worst, float(np.max(np.abs(x[:, s] - xref[:, s])) / rad))
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("subdiv,ncells", [(3, 37), (4, 9)])
def test_noalloc_matches_batched_step_twice(prec, subdiv, ncells):
    """642-vertex cells keep their solve vectors in shared memory; 2562-vertex cells do
    not fit four of them there and keep them in the static workspace."""
    from paper_2011_04332_b300 import native
    b = I.homogeneous_rbc_batch(ncells=ncells, seed=77, velocity_sigma=0.02, subdiv=subdiv)
    n = b.types[0].mesh.n
    assert np.array_equal(b.offsets, np.arange(b.ncells + 1) * n)   # back-to-back layout
    p = native.FP64 if prec == "fp64" else native.FP32FORM
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    ct = native.CellType(b.types[0].mesh.verts, b.types[0].mesh.tris, b.types[0].material.as_tuple(), b.dt)
    batch = native.Batch([ct], b.type_of_cell, p)
    dev = torch.device("cuda:0")
    f = torch.tensor(b.f, dtype=dt_, device=dev)
    iters = torch.tensor(b.iters, device=dev)
    x_in = torch.tensor(b.x, dtype=dt_, device=dev)
    v_in = torch.tensor(b.v, dtype=dt_, device=dev)
    for call in range(2):
        xa, va = x_in.clone(), v_in.clone()
        ra = torch.zeros(b.ncells, dtype=torch.float64, device=dev)
        sa = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
        batch.step(xa, va, f, iters=iters, residual=ra, status=sa)
        xb, vb = x_in.clone(), v_in.clone()
        rb = torch.zeros(b.ncells, dtype=torch.float64, device=dev)
        sb = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
        native.step_noalloc(ct, p, b.ncells, xb, vb, f, iters=iters, residual=rb, status=sb)
        torch.cuda.synchronize()
        xa_, xb_ = xa.double().cpu().numpy(), xb.double().cpu().numpy()
        assert _rel_err(b, xb_, xa_) <= BARS[prec], f"call {call}"
        assert _rel_err(b, vb.double().cpu().numpy() * b.dt, va.double().cpu().numpy() * b.dt,
                        radius_from=xa_) <= BARS[prec], f"call {call}"
        assert torch.equal(sa, sb) and int(sb.min()) >= 0
        assert np.allclose(rb.cpu().numpy(), ra.cpu().numpy(), rtol=1e-4, atol=1e-8)
        # the second call starts from the state the first produced
        x_in, v_in = xa, va


def test_noalloc_rejects_too_many_cells():
    """The library refuses a call beyond its static cell limit before any launch; the
    state tensors are sized for the call, so nothing could go out of bounds even if it
    did not."""
    from paper_2011_04332_b300 import native
    m = I.icosahedron()
    ct = native.CellType(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), 0.1)
    ncells = 65537
    x = torch.zeros(3, ncells * m.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(native.NpfemError) as ei:
        native.step_noalloc(ct, native.FP64, ncells, x, x.clone(), x.clone())
    assert ei.value.code == -6 and "65536" in str(ei.value)


def test_noalloc_wrapper_rejects_mismatched_tensors():
    """The binding checks sizes against ncells before passing pointers to the library."""
    from paper_2011_04332_b300 import native
    m = I.icosahedron()
    ct = native.CellType(m.verts, m.tris, I.RBC_MATERIAL.as_tuple(), 0.1)
    x = torch.zeros(3, 4 * m.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        native.step_noalloc(ct, native.FP64, 5, x, x.clone(), x.clone())          # 4 cells of state, 5 asked
    with pytest.raises(ValueError):
        native.step_noalloc(ct, native.FP32FORM, 4, x, x.clone(), x.clone())     # FP64 tensors, FP32 call
