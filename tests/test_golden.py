"""The stored single-RBC rollout (tests/golden/single_rbc_100_steps.txt, written from the
oracle by tests/golden/make_golden.py): the oracle reproduces it, and the CUDA path lands
on it after 1, 10 and 100 steps in both forms.

Error per quantity = max over the stored vertices of |q - q_ref|_inf / R, R the radius of
the stored positions about their centroid (velocities as v * dt, like positions).  Bars:
the FP64 form repeats the oracle's arithmetic up to the order of its sums, so 100 steps
stay within a few hundred units of FP64 rounding (1.2e-14 measured on B300; bar 1e-12);
the FP32 form stores the state in FP32 (a coordinate rounds by up to 6e-8 of itself each
step) and measured 1.7e-7 after 100 steps (bar 1e-6).  Residuals: FP64 form to 1e-8
relative (7e-11 measured); FP32 form to 2e-2 relative, its gradient norm carrying FP32
noise near 1e-3 of the initial one (2.1e-3 measured).
"""
import importlib.util
import os

import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
G = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(G)

ORACLE_BAR = 1e-11   # the oracle against its own stored output (rounding of another BLAS build)
FP64_BAR = 1e-12
FP32_BAR = 1e-6


def _errors(x, v, xref, vref, dt):
    rad = np.max(np.linalg.norm(xref - xref.mean(axis=1, keepdims=True), axis=0))
    return np.max(np.abs(x - xref)) / rad, np.max(np.abs(v - vref)) * dt / rad


def test_fixture_shape():
    res, st, states, verts = G.read()
    assert sorted(res) == list(range(1, G.NSTEPS + 1))
    assert all(s == O.STATUS_OK for s in st.values())
    assert sorted(states) == list(G.RECORD_STEPS)
    assert np.array_equal(verts, np.arange(0, I.single_rbc().n_total, G.VERTEX_STRIDE))


def test_oracle_reproduces_stored_rollout():
    res, st, states, verts = G.read()
    b, residual, status, got = G.single_rbc_rollout()
    assert status == [st[s] for s in range(1, G.NSTEPS + 1)]
    np.testing.assert_allclose(residual, [res[s] for s in range(1, G.NSTEPS + 1)], rtol=1e-9, atol=0)
    for s in G.RECORD_STEPS:
        ex, ev = _errors(*got[s], *states[s], b.dt)
        assert ex <= ORACLE_BAR and ev <= ORACLE_BAR, (s, ex, ev)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cuda_rollout_lands_on_stored_rollout(prec):
    """100 steps on the GPU from the stored start, no oracle in the loop: positions and
    velocities of the stored vertices after steps 1, 10 and 100, every step's status and
    residual."""
    import torch
    from paper_2011_04332_b300 import native as nat
    res, st, states, verts = G.read()
    b = I.single_rbc()
    precision = nat.FP64 if prec == "fp64" else nat.FP32FORM
    dtype = torch.float64 if prec == "fp64" else torch.float32
    bar = FP64_BAR if prec == "fp64" else FP32_BAR
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    batch = nat.Batch(types, b.type_of_cell, precision)
    dev = torch.device("cuda:0")
    X = torch.tensor(b.x, dtype=dtype, device=dev).contiguous()
    V = torch.tensor(b.v, dtype=dtype, device=dev).contiguous()
    F = torch.tensor(b.f, dtype=dtype, device=dev).contiguous()
    it = torch.tensor(b.iters, device=dev)
    r = torch.empty(1, dtype=torch.float64, device=dev)
    s_out = torch.empty(1, dtype=torch.int32, device=dev)
    for s in range(1, G.NSTEPS + 1):
        batch.step(X, V, F, iters=it, residual=r, status=s_out)
        torch.cuda.synchronize()
        assert int(s_out.item()) == st[s], s
        assert float(r.item()) == pytest.approx(res[s], rel=1e-8 if prec == "fp64" else 2e-2), s
        if s in states:
            x = X.double().cpu().numpy()[:, verts]
            v = V.double().cpu().numpy()[:, verts]
            ex, ev = _errors(x, v, *states[s], b.dt)
            assert ex <= bar and ev <= bar, (s, ex, ev)
