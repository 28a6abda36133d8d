"""The membrane-calibration workload at full size: 256 placed 642-vertex RBCs (FP64),
checkpoints every 20 steps inside the library's rollout adjoint, and the diameter loss
of 8 cells (the adjoint's use case: calibrating membrane parameters against target
deformations, Setting up new materials section).

* The 200-step rollout adjoint equals, bit for bit, the chain of 200 single-step
  adjoints run on the stored forward states (the checkpointing recomputes the same
  states), and its per-type weight gradients equal the chain's sums to rounding.
* Central differences (relative step 1e-6) of the loss after 100 steps agree with the
  adjoint to 1e-6 for the four material weights.  Along the force field itself and along
  random affine fields per cell of the forces and of the initial positions (of the
  field's own RMS size, or 0.1 um for positions) they agree to 1e-6 as well, taken at
  h = 4e-5, 2e-5 and 1e-5 and extrapolated twice (removing the h^2 and h^4 terms): at
  h <= 2e-6 the loss's own rounding (about 1e-12 of a loss of 3e3, after 100 FP64 steps)
  divided by the step is already 1e-6 of the smallest of these derivatives (measured:
  the initial-position direction's plain differences lie 1.0e-6 .. 1.3e-6 from the
  adjoint for h = 2e-6 .. 5e-7, the twice-extrapolated ones 1e-8 from it).  After 10
  steps also along the gradient's own per-vertex fields (h = 1e-6 and 5e-7, extrapolated
  once).  Along white-noise directions the loss is strongly nonlinear at
  longer horizons: after 100 steps the central differences converge to the
  adjoint only as h^2 (relative error 1.5e-4 at h = 1e-6, 2e-6 at 1e-7).  After 200
  steps the loss is too nonlinear for central differences to serve as a reference at
  all: at steps 1e-4 ... 1e-7 they scatter (91, -1259, 216, 214 for the strain weight,
  adjoint 214.12) with every line-search step length unchanged, while at 10, 50 and 100
  steps they agree with the adjoint to 1e-7.
"""
import numpy as np
import pytest

from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCELLS, CKPT = 256, 20
CELLS = np.arange(0, NCELLS, NCELLS // 8)      # the 8 cells whose diameters enter the loss
H = 1e-6
H_DIR = 4e-5                                  # largest step of the directional checks after 100 steps


@pytest.fixture(scope="module")
def setup():
    from paper_2011_04332_b300 import autograd as AG
    b = I.homogeneous_rbc_batch(ncells=NCELLS, seed=1003)
    rng = np.random.default_rng(1003)
    targets = rng.uniform(6.0, 12.0, size=(NCELLS, 2))
    cal = AG.Calibration(b.types[0].mesh, b.types[0].material.as_tuple(), b.dt, NCELLS)
    return b, targets, cal


def _diameter_loss_grad(cal, xN, targets):
    """Loss of the 8 cells and its gradient with respect to x_N."""
    from paper_2011_04332_b300 import autograd as AG
    xg = xN.detach().clone().requires_grad_(True)
    D = AG.diameters(xg, cal.offsets, cal.sets)
    sel = torch.as_tensor(CELLS, device=xg.device)
    loss = ((D[sel] - targets[sel]) ** 2).sum()
    loss.backward()
    return float(loss), xg.grad.contiguous()


def _loss_of(cal, b, x0, v0, f, targets, iters, nsteps, weights=None):
    """Loss of the 8 cells after an nsteps rollout (no gradient), optionally with new weights."""
    if weights is not None:
        cal.rebuild(np.asarray(list(weights) + [b.types[0].material.density]))
    x, v = x0.clone(), v0.clone()
    for _ in range(nsteps):
        cal.batch.step(x, v, f, iters=iters)
    return _diameter_loss_grad(cal, x, targets)[0]


def test_rollout_adjoint_equals_step_chain_at_200_steps(setup):
    b, targets_np, cal = setup
    dev = torch.device("cuda:0")
    nsteps = 200
    cal.rebuild(np.asarray(list(b.types[0].material.as_tuple()[:4]) + [b.types[0].material.density]))
    batch = cal.batch
    x0, v0, f = (torch.tensor(a, device=dev) for a in (b.x, b.v, b.f))
    iters = torch.tensor(b.iters, device=dev)
    targets = torch.tensor(targets_np, device=dev)
    xs, vs = [x0.clone()], [v0.clone()]
    for _ in range(nsteps):
        x, v = xs[-1].clone(), vs[-1].clone()
        batch.step(x, v, f, iters=iters)
        xs.append(x)
        vs.append(v)
    _, gxe = _diameter_loss_grad(cal, xs[-1], targets)
    gx, gv, gf = (torch.empty_like(x0) for _ in range(3))
    gw = torch.empty((1, 4), dtype=torch.float64, device=dev)
    st = torch.full((NCELLS,), -1, dtype=torch.int32, device=dev)
    batch.rollout_adjoint(x0, v0, f, gxe, None, gx, gv, gf, gw, nsteps, CKPT, iters=iters, status=st)
    cx, cv, cf = gxe.clone(), torch.zeros_like(x0), torch.zeros_like(x0)
    cw = torch.zeros((NCELLS, 4), dtype=torch.float64, device=dev)
    for s in range(nsteps - 1, -1, -1):
        nx, nv, nf = (torch.empty_like(x0) for _ in range(3))
        gwc = torch.empty((NCELLS, 4), dtype=torch.float64, device=dev)
        batch.step_adjoint(xs[s], vs[s], f, cx, cv, nx, nv, nf, gwc, iters=iters)
        cx, cv = nx, nv
        cf += nf
        cw += gwc
    torch.cuda.synchronize()
    assert torch.equal(gx, cx) and torch.equal(gv, cv) and torch.equal(gf, cf)
    assert torch.allclose(gw[0], cw.sum(dim=0), rtol=1e-12, atol=0)
    assert int(st.max()) == 0 and int(st.min()) == 0
    # the forward states of the rollout equal the recomputed chain: the loss is finite and
    # its gradient reaches the initial state
    assert torch.isfinite(gx).all() and float(gx.abs().max()) > 0.0


def test_calibration_gradient_matches_central_differences(setup):
    from paper_2011_04332_b300 import autograd as AG
    b, targets_np, cal = setup
    nsteps = 100
    dev = torch.device("cuda:0")
    w0 = np.array(b.types[0].material.as_tuple()[:4])
    cal.rebuild(np.asarray(list(w0) + [b.types[0].material.density]))
    x0 = torch.tensor(b.x, device=dev, requires_grad=True)
    v0 = torch.tensor(b.v, device=dev)
    f = torch.tensor(b.f, device=dev, requires_grad=True)
    iters = torch.tensor(b.iters, device=dev)
    targets = torch.tensor(targets_np, device=dev)
    w = torch.tensor([cal.material[:4]], dtype=torch.float64, device=dev, requires_grad=True)
    toc = torch.zeros(NCELLS, dtype=torch.int32, device=dev)
    xN, _ = AG.rollout(cal.batch, x0, v0, f, w, toc, iters, nsteps, CKPT)
    D = AG.diameters(xN, cal.offsets, cal.sets)
    sel = torch.as_tensor(CELLS, device=dev)
    loss = ((D[sel] - targets[sel]) ** 2).sum()
    loss.backward()
    gw = w.grad.cpu().numpy()[0]
    gf, gx = f.grad, x0.grad
    # gradients vanish outside the 8 cells (cells are independent)
    mask = torch.zeros(b.n_total, dtype=torch.bool, device=dev)
    for c in CELLS:
        mask[int(b.offsets[c]):int(b.offsets[c + 1])] = True
    assert float(gf[:, ~mask].abs().max()) == 0.0 and float(gf[:, mask].abs().max()) > 0.0

    # material weights: central differences of the rebuilt type, relative step H; each
    # component within 1e-6 of the gradient's norm (a component near zero is otherwise
    # judged on the differences' own rounding noise)
    fd = np.zeros(4)
    for q in range(4):
        hq = H * w0[q]
        wp, wm = w0.copy(), w0.copy()
        wp[q] += hq
        wm[q] -= hq
        lp = _loss_of(cal, b, x0.detach(), v0, f.detach(), targets, iters, nsteps, wp)
        lm = _loss_of(cal, b, x0.detach(), v0, f.detach(), targets, iters, nsteps, wm)
        fd[q] = (lp - lm) / (2 * hq)
    cal.rebuild(np.asarray(list(w0) + [b.types[0].material.density]))
    assert np.max(np.abs(gw - fd)) <= 1e-6 * np.linalg.norm(gw), (gw, fd)

    # directions of the forces and of the initial positions (step H relative to the field)
    rng = np.random.default_rng(7)
    frms = float(f.detach().pow(2).mean().sqrt())
    for name, d in (("f along itself", f.detach().clone()),
                    ("f affine", _unit_rms(_affine_field(b, rng)) * frms),
                    ("x0 affine", _unit_rms(_affine_field(b, rng)) * 0.1)):
        grad = gf if name.startswith("f") else gx
        fd_ = _central_difference(cal, b, x0.detach(), v0, f.detach(), targets, iters, nsteps, name[0], d,
                                  h=H_DIR, levels=3)
        adj = float((grad * d).sum())
        assert adj == pytest.approx(fd_, rel=1e-6), (name, adj, fd_)


def test_gradient_directions_after_10_steps(setup):
    """Central differences along the adjoint's own gradient fields of the forces and of
    the initial positions (per-vertex, white-noise-like fields over the 8 cells; the
    direction of the largest directional derivative, so it stands far above the
    differences' rounding noise, unlike a random direction nearly orthogonal to it)."""
    from paper_2011_04332_b300 import autograd as AG
    b, targets_np, cal = setup
    nsteps = 10
    dev = torch.device("cuda:0")
    cal.rebuild(np.asarray(list(b.types[0].material.as_tuple()[:4]) + [b.types[0].material.density]))
    x0 = torch.tensor(b.x, device=dev, requires_grad=True)
    v0 = torch.tensor(b.v, device=dev)
    f = torch.tensor(b.f, device=dev, requires_grad=True)
    iters = torch.tensor(b.iters, device=dev)
    targets = torch.tensor(targets_np, device=dev)
    w = torch.tensor([cal.material[:4]], dtype=torch.float64, device=dev, requires_grad=True)
    toc = torch.zeros(NCELLS, dtype=torch.int32, device=dev)
    xN, _ = AG.rollout(cal.batch, x0, v0, f, w, toc, iters, nsteps, CKPT)
    D = AG.diameters(xN, cal.offsets, cal.sets)
    sel = torch.as_tensor(CELLS, device=dev)
    ((D[sel] - targets[sel]) ** 2).sum().backward()
    for which, grad, scale in (("f", f.grad, float(f.detach().abs().max())), ("x", x0.grad, 1.0)):
        d = grad / float(grad.abs().max()) * scale
        fd_ = _central_difference(cal, b, x0.detach(), v0, f.detach(), targets, iters, nsteps, which, d)
        adj = float((grad * d).sum())
        assert adj == pytest.approx(fd_, rel=1e-6), (which, adj, fd_)


def _unit_rms(d):
    return d / float(d.pow(2).mean().sqrt())


def _affine_field(b, rng):
    """A random affine field per cell, A_c (x - c) + t_c with the cell's rest centroid c
    (a smooth direction: stretches, shears, rotations and translations of each cell)."""
    out = np.empty_like(b.x)
    for c in range(b.ncells):
        s = b.cell_slice(c)
        xc = b.x[:, s]
        ctr = xc.mean(axis=1, keepdims=True)
        out[:, s] = rng.standard_normal((3, 3)) @ (xc - ctr) / 4.0 + rng.standard_normal((3, 1))
    return torch.tensor(out, device="cuda:0")


def _central_difference(cal, b, x0, v0, f, targets, iters, nsteps, which, d, h=H, levels=2):
    """Central differences D along d, Richardson-extrapolated.  levels=2: steps h and h/2,
    (4 D(h/2) - D(h))/3, which removes the h^2 error term; levels=3: steps h, h/2, h/4,
    (64 D(h/4) - 20 D(h/2) + D(h))/45, which removes the h^2 and h^4 terms."""
    def cd(s):
        if which == "f":
            lp = _loss_of(cal, b, x0, v0, f + s * d, targets, iters, nsteps)
            lm = _loss_of(cal, b, x0, v0, f - s * d, targets, iters, nsteps)
        else:
            lp = _loss_of(cal, b, x0 + s * d, v0, f, targets, iters, nsteps)
            lm = _loss_of(cal, b, x0 - s * d, v0, f, targets, iters, nsteps)
        return (lp - lm) / (2 * s)
    if levels == 2:
        return (4.0 * cd(h / 2) - cd(h)) / 3.0
    assert levels == 3
    return (64.0 * cd(h / 4) - 20.0 * cd(h / 2) + cd(h)) / 45.0


def test_rollout_adjoint_sums_weight_gradients_per_type():
    """A two-type batch: the rollout adjoint's per-type weight gradients equal the sums
    of the per-cell step-adjoint gradients of a step-by-step chain."""
    from paper_2011_04332_b300 import native
    dev = torch.device("cuda:0")
    b = I.heterogeneous_batch(n_rbc3=3, n_rbc4=0, n_plt=4, seed=21, iters_range=(2, 5))
    present = sorted(set(int(t) for t in b.type_of_cell))
    types = [native.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    batch = native.Batch(types, b.type_of_cell, native.FP64)
    x0, v0, f = (torch.tensor(a, device=dev) for a in (b.x, b.v, b.f))
    iters = torch.tensor(b.iters, device=dev)
    rng = np.random.default_rng(5)
    gxe = torch.tensor(rng.standard_normal(b.x.shape), device=dev)
    gve = torch.tensor(rng.standard_normal(b.x.shape), device=dev)
    nsteps, ckpt = 5, 2
    gx, gv, gf = (torch.empty_like(x0) for _ in range(3))
    gw = torch.full((len(types), 4), np.nan, dtype=torch.float64, device=dev)
    st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
    batch.rollout_adjoint(x0, v0, f, gxe, gve, gx, gv, gf, gw, nsteps, ckpt, iters=iters, status=st)
    # chain: states by forward steps, then the step adjoints in reverse
    xs, vs = [x0.clone()], [v0.clone()]
    for _ in range(nsteps - 1):
        x, v = xs[-1].clone(), vs[-1].clone()
        batch.step(x, v, f, iters=iters)
        xs.append(x)
        vs.append(v)
    cx, cv, cf = gxe.clone(), gve.clone(), torch.zeros_like(x0)
    cw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    for s in range(nsteps - 1, -1, -1):
        nx, nv, nf = (torch.empty_like(x0) for _ in range(3))
        gwc = torch.empty((b.ncells, 4), dtype=torch.float64, device=dev)
        batch.step_adjoint(xs[s], vs[s], f, cx, cv, nx, nv, nf, gwc, iters=iters)
        cx, cv = nx, nv
        cf += nf
        cw += gwc
    torch.cuda.synchronize()
    assert torch.equal(gx, cx) and torch.equal(gv, cv) and torch.equal(gf, cf)
    toc = torch.tensor(b.type_of_cell, device=dev).long()
    for t in range(len(types)):
        want = cw[toc == t].sum(dim=0)
        if t not in present:
            assert float(gw[t].abs().max()) == 0.0
        else:
            assert torch.allclose(gw[t], want, rtol=1e-13, atol=0), (t, gw[t], want)
    assert int(st.min()) == 0 and int(st.max()) == 0
