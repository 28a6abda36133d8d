"""GPU reverse mode of the step (npfem_step_adjoint) against two independent references:

* the oracle's own forward-mode derivative (complex step through the whole FP64 oracle
  step): the dot-product identity lambda^T (J delta) = (J^T lambda)^T delta with random
  delta over (x_n, v_n, f, weights) and random lambda over (x_{n+1}, v_{n+1});
* central finite differences of the GPU forward step (h = 1e-6 relative).
"""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H_CS = 1e-30


def _native():
    from paper_2011_04332_b300 import native
    return native


def gpu_adjoint(b, lam_x, lam_v, iters=None, damping=()):
    nat = _native()
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple() + tuple(damping), b.dt)
             for t in b.types]
    batch = nat.Batch(types, b.type_of_cell, nat.FP64)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, v, f = T(b.x), T(b.v), T(b.f)
    gxn, gvn = T(lam_x), T(lam_v)
    gx, gv, gf = torch.zeros_like(x), torch.zeros_like(x), torch.zeros_like(x)
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
    it = torch.tensor(b.iters if iters is None else iters, device=dev)
    batch.step_adjoint(x, v, f, gxn, gvn, gx, gv, gf, gw, iters=it, status=st)
    torch.cuda.synchronize()
    assert int(st.max()) == 0 and int(st.min()) == 0
    return (gx.cpu().numpy(), gv.cpu().numpy(), gf.cpu().numpy(), gw.cpu().numpy())


def oracle_jvp(b, dx, dv, df, dws, damping=()):
    """Complex-step J.delta of (x_{n+1}, v_{n+1}); dws[type] perturbs the weight scale;
    damping = (c_alpha, c_beta) joins every type's material."""
    out_x = np.zeros_like(b.x)
    out_v = np.zeros_like(b.x)
    for c in range(b.ncells):
        t = int(b.type_of_cell[c])
        spec = b.types[t]
        ws = np.ones(4, complex) + 1j * H_CS * dws[t]
        ct = O.CellType(spec.mesh.verts, spec.mesh.tris, spec.material.as_tuple() + tuple(damping), b.dt, ws)
        s = b.cell_slice(c)
        x = b.x[:, s].T + 1j * H_CS * dx[:, s].T
        v = b.v[:, s].T + 1j * H_CS * dv[:, s].T
        f = b.f[:, s].T + 1j * H_CS * df[:, s].T
        r = O.step(ct.rest, ct.solver, x, v, f, int(b.iters[c]), ws)
        out_x[:, s] = (np.imag(r.x) / H_CS).T
        out_v[:, s] = (np.imag(r.v) / H_CS).T
    return out_x, out_v


@pytest.mark.parametrize("seed,damping", [(3, ()), (4, ()), (5, (0.5, 1.0))])
def test_adjoint_dot_product_against_oracle_forward_mode(seed, damping):
    """Without and with Rayleigh damping (whose dissipation term makes every iterate's
    gradient depend on x_n directly)."""
    b = I.small_mixed_batch(seed=seed, iters=(3, 6))
    rng = np.random.default_rng(seed)
    lam_x = rng.standard_normal(b.x.shape)
    lam_v = rng.standard_normal(b.x.shape) * 1e-2
    dx = rng.standard_normal(b.x.shape) * 1e-2
    dv = rng.standard_normal(b.x.shape) * 1e-2
    df = rng.standard_normal(b.x.shape) * 1e-3
    dws = rng.standard_normal((len(b.types), 4))
    jx, jv = oracle_jvp(b, dx, dv, df, dws, damping)
    lhs = np.sum(lam_x * jx) + np.sum(lam_v * jv)
    gx, gv, gf, gw = gpu_adjoint(b, lam_x, lam_v, damping=damping)
    rhs = np.sum(gx * dx) + np.sum(gv * dv) + np.sum(gf * df)
    for c in range(b.ncells):
        t = int(b.type_of_cell[c])
        wmat = np.array(b.types[t].material.as_tuple()[:4])
        rhs += np.sum(gw[c] * wmat * dws[t])      # d/d(scale) = w * d/dw
    assert rhs == pytest.approx(lhs, rel=1e-9)
    # each input block separately (catches compensating errors)
    for blk in range(4):
        d = [np.zeros_like(dx), np.zeros_like(dv), np.zeros_like(df), np.zeros_like(dws)]
        d[blk] = [dx, dv, df, dws][blk]
        jx, jv = oracle_jvp(b, *d, damping=damping)
        l2 = np.sum(lam_x * jx) + np.sum(lam_v * jv)
        r2 = np.sum(gx * d[0]) + np.sum(gv * d[1]) + np.sum(gf * d[2])
        for c in range(b.ncells):
            t = int(b.type_of_cell[c])
            r2 += np.sum(gw[c] * np.array(b.types[t].material.as_tuple()[:4]) * d[3][t])
        assert r2 == pytest.approx(l2, rel=1e-8, abs=1e-12 * abs(lhs)), f"block {blk}"


def test_adjoint_launch_shapes_agree():
    """The unrolled adjoint (a CTA of four warps per cell over the launch's warp slots)
    gives the same bits whatever the launch shape: the solve vector in shared memory or in
    the workspace (the path of types whose vectors do not fit, such as 2562 vertices), the
    three coordinates swept together or one after another, and 1 to 4 warp slots per CTA
    of the step (other slot counts and CTA grids).  Damped, so every term is exercised."""
    nat = _native()
    b = I.small_mixed_batch(seed=11, iters=(2, 5))
    damping = (0.5, 1.0)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple() + damping, b.dt) for t in b.types]
    batch = nat.Batch(types, b.type_of_cell, nat.FP64)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    rng = np.random.default_rng(11)
    x, v, f = T(b.x), T(b.v), T(b.f)
    gxn, gvn = T(rng.standard_normal(b.x.shape)), T(rng.standard_normal(b.x.shape) * 1e-2)
    it = torch.tensor(b.iters, device=dev)

    def run():
        gx, gv, gf = torch.zeros_like(x), torch.zeros_like(x), torch.zeros_like(x)
        gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
        st = torch.full((b.ncells,), -1, dtype=torch.int32, device=dev)
        batch.step_adjoint(x, v, f, gxn, gvn, gx, gv, gf, gw, iters=it, status=st)
        torch.cuda.synchronize()
        assert int(st.max()) == 0 and int(st.min()) == 0
        return [a.cpu().numpy() for a in (gx, gv, gf, gw)]

    ref = run()
    assert all(np.isfinite(a).all() for a in ref) and np.abs(ref[3]).max() > 0
    for wpb, bps, shared, per_coord in ((4, 3, False, False), (4, 3, True, True), (1, 8, True, False),
                                        (2, 2, False, True)):
        for t in range(len(types)):
            batch.set_launch(t, wpb, bps, shared, per_coord)
        out = run()
        for a, c in zip(ref, out):
            assert np.array_equal(a, c), (wpb, bps, shared, per_coord)


def test_adjoint_matches_central_differences_rbc642():
    """Eight placed 642-vertex RBCs (the calibration workload's cells), FP64: the adjoint
    of L = lambda.v_{n+1} w.r.t. forces and the four weights against central differences
    of the GPU forward step (h = 1e-6 relative).  The loss uses the velocity output,
    which carries no absolute-position rounding (positions near 100 um would put
    ~1e-12 of rounding into a sum over 15k terms and swamp the difference quotient)."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=8, seed=1003, velocity_sigma=0.02)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal(b.x.shape)
    gx, gv, gf, gw = gpu_adjoint(b, np.zeros_like(lam), lam)
    dev = torch.device("cuda:0")

    def loss(f=None, mat=None):
        mats = [t.material.as_tuple() if mat is None else mat for t in b.types]
        types = [nat.CellType(t.mesh.verts, t.mesh.tris, m, b.dt) for t, m in zip(b.types, mats)]
        bt = nat.Batch(types, b.type_of_cell, nat.FP64)
        x = torch.tensor(b.x, device=dev)
        v = torch.tensor(b.v, device=dev)
        ff = torch.tensor(b.f if f is None else f, device=dev)
        al = torch.zeros((b.ncells, 8), dtype=torch.float64, device=dev)
        bt.step(x, v, ff, iters=torch.tensor(b.iters, device=dev), alpha_log=al)
        torch.cuda.synchronize()
        return float(np.sum(lam * v.cpu().numpy())), al.cpu().numpy()

    _, al0 = loss()
    # forces, along a random direction
    df = rng.standard_normal(b.f.shape) * np.abs(b.f).max()
    h = 1e-6
    lp, alp = loss(f=b.f + h * df)
    lm, alm = loss(f=b.f - h * df)
    assert np.array_equal(alp, al0) and np.array_equal(alm, al0)
    fd = (lp - lm) / (2 * h)
    assert np.sum(gf * df) == pytest.approx(fd, rel=1e-6)
    # weights (all cells share the type).  Bar: 1e-6 relative to the largest weight
    # derivative; the area and volume derivatives are small enough that the quotient's
    # own rounding (~1e-9) is comparable to 1e-6 of their value.
    base = np.array(b.types[0].material.as_tuple())
    gscale = np.max(np.abs(gw.sum(axis=0)))
    for q in range(4):
        hq = h * base[q]
        mp, mm = base.copy(), base.copy()
        mp[q] += hq
        mm[q] -= hq
        lp, _ = loss(mat=tuple(mp))
        lm, _ = loss(mat=tuple(mm))
        fd = (lp - lm) / (2 * hq)
        assert abs(np.sum(gw[:, q]) - fd) <= 1e-6 * gscale, f"weight {q}"


def test_adjoint_rejects_fp32_batches_and_long_iterations():
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=2, seed=5)
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    bt = nat.Batch(types, b.type_of_cell, nat.FP32FORM)
    x = torch.zeros(3, b.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.NpfemError):
        bt.step_adjoint(x, x, x, x, x, x, x, x, torch.zeros(2, 4, dtype=torch.float64, device="cuda"))
    b64 = nat.Batch(types, b.type_of_cell, nat.FP64)
    st = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    it = torch.tensor([17, 3], dtype=torch.int32, device="cuda")
    xs = torch.tensor(b.x, device="cuda")
    g = torch.zeros_like(xs)
    b64.step_adjoint(xs, g, g, g, g, g.clone(), g.clone(), g.clone(),
                     torch.zeros(2, 4, dtype=torch.float64, device="cuda"), iters=it, status=st)
    torch.cuda.synchronize()
    assert st.tolist() == [8, 0]
