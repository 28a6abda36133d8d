"""Checkpointed rollout gradients (torch.autograd over npfem_step_adjoint) for the
membrane-calibration loss, against the oracle's complex-step directional derivative
of the same loss through the same rollout, and the checkpointing against a plain
step-by-step chain of StepFunction."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H_CS = 1e-30


def _setup(ncells=8, seed=1003):
    b = I.homogeneous_rbc_batch(ncells=ncells, seed=seed, subdiv=2, velocity_sigma=0.01)
    rng = np.random.default_rng(seed)
    targets = rng.uniform(6.0, 12.0, size=(ncells, 2))
    return b, targets


def _oracle_loss(b, targets, nsteps, f, ws, sets):
    spec = b.types[0]
    ct = O.CellType(spec.mesh.verts, spec.mesh.tris, spec.material.as_tuple(), b.dt, ws)
    loss = 0.0
    (ax0, ax1), (tr0, tr1) = sets
    for c in range(b.ncells):
        s = b.cell_slice(c)
        x, v = b.x[:, s].T.astype(complex), b.v[:, s].T.astype(complex)
        fc = f[:, s].T
        for _ in range(nsteps):
            r = O.step(ct.rest, ct.solver, x, v, fc, int(b.iters[c]), ws)
            x, v = r.x, r.v
        for q, (i0, i1) in enumerate(((ax0, ax1), (tr0, tr1))):
            d = x[i1].mean(axis=0) - x[i0].mean(axis=0)
            D = np.sqrt(np.sum(d * d))
            loss = loss + (D - targets[c, q]) ** 2
    return loss


def test_rollout_gradient_matches_oracle_complex_step():
    from paper_2011_04332_b300 import autograd as AG
    b, targets = _setup()
    nsteps, ckpt = 10, 4
    cal = AG.Calibration(b.types[0].mesh, b.types[0].material.as_tuple(), b.dt, b.ncells)
    dev = torch.device("cuda:0")
    x0 = torch.tensor(b.x, device=dev)
    v0 = torch.tensor(b.v, device=dev)
    f = torch.tensor(b.f, device=dev, requires_grad=True)
    iters = torch.tensor(b.iters, device=dev)
    loss, w = cal.loss(x0, v0, f, torch.tensor(targets, device=dev), iters, nsteps, ckpt)
    loss.backward()
    gf, gw = f.grad.cpu().numpy(), w.grad.cpu().numpy()[0]
    rng = np.random.default_rng(2)
    df = rng.standard_normal(b.f.shape) * 1e-3
    dws = rng.standard_normal(4)
    mat = np.array(b.types[0].material.as_tuple()[:4])
    lc = _oracle_loss(b, targets, nsteps, b.f + 1j * H_CS * df, np.ones(4) + 1j * H_CS * dws, cal.sets)
    dl_ref = np.imag(lc) / H_CS
    dl_gpu = np.sum(gf * df) + np.sum(gw * mat * dws)
    assert float(np.real(lc)) == pytest.approx(float(loss.detach()), rel=1e-10)
    assert dl_gpu == pytest.approx(dl_ref, rel=1e-8)


def test_checkpointed_rollout_equals_step_chain():
    from paper_2011_04332_b300 import autograd as AG
    from paper_2011_04332_b300 import native
    b, targets = _setup(ncells=4, seed=7)
    dev = torch.device("cuda:0")
    cal = AG.Calibration(b.types[0].mesh, b.types[0].material.as_tuple(), b.dt, b.ncells)
    iters = torch.tensor(b.iters, device=dev)
    tg = torch.tensor(targets, device=dev)
    grads = []
    for mode in ("rollout", "chain"):
        x = torch.tensor(b.x, device=dev, requires_grad=True)
        v = torch.tensor(b.v, device=dev, requires_grad=True)
        f = torch.tensor(b.f, device=dev, requires_grad=True)
        w = torch.tensor([cal.material[:4]], dtype=torch.float64, device=dev, requires_grad=True)
        toc = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
        if mode == "rollout":
            xN, vN = AG.rollout(cal.batch, x, v, f, w, toc, iters, 7, 3)
        else:
            xN, vN = x, v
            for _ in range(7):
                xN, vN = AG.step(cal.batch, xN, vN, f, w, toc, iters)
        D = AG.diameters(xN, cal.offsets, cal.sets)
        loss = ((D - tg) ** 2).sum() + (vN ** 2).sum()
        loss.backward()
        grads.append([t.grad.cpu().numpy() for t in (x, v, f, w)])
    for a, c in zip(*grads):
        assert np.allclose(a, c, rtol=1e-12, atol=1e-12 * np.max(np.abs(c)))
    del native
