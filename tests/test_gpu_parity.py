"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle, one step
from identical inputs, element by element on vertex positions and velocities.

Bars (error per cell = max_j |x_j - x_j^ref|_inf / max_j |x_j^ref - centroid^ref|):
  FP64 form        <= 1e-10
  FP32 form        <= 1e-5   (FP32 local work, FP64 factor/solves/reductions)
The accepted line-search step lengths are integers in disguise (a count of halvings)
and are compared exactly in the FP64 form.
"""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
FP32_BAR = 1e-5


def _native():
    from paper_2011_04332_b300 import native
    return native


class Runner:
    """Builds library types/batch for a BatchInputs and steps it on the GPU."""

    def __init__(self, b: I.BatchInputs, precision: int):
        nat = _native()
        self.b = b
        self.prec = precision
        self.types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
        self.batch = nat.Batch(self.types, b.type_of_cell, precision)
        assert self.batch.n_total == b.n_total
        assert np.array_equal(self.batch.offsets, b.offsets)
        self.dtype = torch.float64 if precision == nat.FP64 else torch.float32

    def step(self, x, v, f, iters=None, alpha_len=8, iters_default=5, max_iters=0):
        dev = torch.device("cuda:0")
        X = torch.tensor(x, dtype=self.dtype, device=dev).contiguous()
        Vt = torch.tensor(v, dtype=self.dtype, device=dev).contiguous()
        F = torch.tensor(f, dtype=self.dtype, device=dev).contiguous()
        it = None if iters is None else torch.tensor(np.asarray(iters, np.int32), device=dev)
        nc = self.b.ncells
        res = torch.full((max(nc, 1),), -1.0, dtype=torch.float64, device=dev)
        st = torch.full((max(nc, 1),), -1, dtype=torch.int32, device=dev)
        al = torch.zeros((max(nc, 1), alpha_len), dtype=torch.float64, device=dev)
        self.batch.step(X, Vt, F, iters=it, iters_default=iters_default, residual=res, status=st, alpha_log=al,
                        max_iters=max_iters)
        torch.cuda.synchronize()
        return (X.double().cpu().numpy(), Vt.double().cpu().numpy(), res.cpu().numpy()[:nc],
                st.cpu().numpy()[:nc], al.cpu().numpy()[:nc])


def oracle_types(b: I.BatchInputs):
    return [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]


def cell_errors(b, x, xref, radius_from=None):
    """Per-cell max-norm error divided by the cell radius (of `radius_from`, default xref)."""
    errs = []
    rf = xref if radius_from is None else radius_from
    for c in range(b.ncells):
        s = b.cell_slice(c)
        xr = rf[:, s]
        rad = np.max(np.linalg.norm(xr - xr.mean(axis=1, keepdims=True), axis=0))
        errs.append(np.max(np.abs(x[:, s] - xref[:, s])) / rad)
    return np.array(errs)


def compare(b, precision, cells=None, steps=1, iters=None, check_alpha=True, bar=None, shapes=None, width=None):
    nat = _native()
    r = Runner(b, precision)
    for t, shape in (shapes or {}).items():
        r.batch.set_split_launch(t, shape)
    if width is not None:
        for t in range(len(b.types)):
            r.batch.set_iter_width(t, width)
    ots = oracle_types(b)
    x, v, f = b.x.copy(), b.v.copy(), b.f.copy()
    if precision == nat.FP32FORM:
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    iters = b.iters if iters is None else iters
    bar = bar if bar is not None else (FP64_BAR if precision == nat.FP64 else FP32_BAR)
    worst = 0.0
    for s in range(steps):
        xg, vg, res, st, al = r.step(x, v, f, iters=iters)
        ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, iters, cells=cells)
        sel = list(range(b.ncells)) if cells is None else list(cells)
        e = cell_errors(b, xg, ref["x"])[sel]
        ev = cell_errors(b, vg * b.dt, ref["v"] * b.dt, radius_from=ref["x"])[sel]
        worst = max(worst, float(e.max()), float(ev.max()))
        assert e.max() <= bar, f"step {s}: position error {e.max():.3e} > {bar}"
        assert ev.max() <= bar, f"step {s}: velocity*dt error {ev.max():.3e} > {bar}"
        for c in sel:
            assert st[c] == ref["status"][c]
            if check_alpha and precision == nat.FP64:
                n_it = int(iters[c])
                assert np.array_equal(al[c, :min(n_it, al.shape[1])], np.array(ref["alphas"][c][:al.shape[1]]))
            if precision == nat.FP64:
                assert res[c] == pytest.approx(ref["residual"][c], rel=1e-4, abs=1e-8)
        # next step from the oracle's state so that both sides see identical inputs
        x, v = ref["x"], ref["v"]
        if precision == nat.FP32FORM:
            x, v = (a.astype(np.float32).astype(np.float64) for a in (x, v))
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_rbc_parity(prec):
    """Single 642-vertex Evans-Fung RBC, axial 10 pN stretch + 0.1 pN noise, 5 iterations,
    three consecutive steps (each from the oracle's previous state)."""
    nat = _native()
    b = I.single_rbc()
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM, steps=3)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_mixed_batch_parity(prec):
    """Three small types (42-vertex RBC, 42-vertex platelet, 162-vertex RBC), ragged
    per-cell iteration counts, non-zero initial velocities."""
    nat = _native()
    b = I.small_mixed_batch()
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM, steps=2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_homogeneous_batch_parity(prec):
    """48 placed 642-vertex RBCs (random rotation, translation in a 200 um box,
    Gaussian + linear-shear forces): more cells than warps per block, ragged tail."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=48, seed=1001, velocity_sigma=0.02)
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_batch_sampled_cells(prec):
    """The 4096-cell homogeneous workload in the benchmark's launch configuration;
    16 sampled cells are checked against the oracle."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=4096, seed=1001)
    cells = sorted(np.random.default_rng(5).choice(4096, size=16, replace=False).tolist())
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM, cells=cells)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stress_mix_sampled_cells(prec):
    """The 20000-cell serving-shaped mix (70 % 642-vertex RBC, 10 % 2562-vertex RBC, 20 %
    platelets) with the default launch shapes: 32 sampled cells against the oracle, for the
    first step and for a step under a re-drawn force field."""
    nat = _native()
    precision = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = I.stress_mix_batch()
    cells = sorted(np.random.default_rng(11).choice(b.ncells, size=32, replace=False).tolist())
    compare(b, precision, cells=cells)
    b.f = I.redrawn_forces(b, b.x, 1005, 1)
    compare(b, precision, cells=cells)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_10k_batch_sampled_cells(prec):
    """The mixed 10^4-cell batch of the benchmark (4500 642-vertex RBCs, 4500 2562-vertex
    RBCs and 1000 platelets in a seeded random order, 3..8 iterations per cell) in its
    default launch configuration (concurrent chains per type, CTA iteration kernels in
    the FP32 form): 5 sampled cells of every type against the oracle, positions,
    velocities, statuses, residuals and (FP64) the accepted step lengths."""
    nat = _native()
    b = I.heterogeneous_batch(4500, 4500, 1000, seed=1002)
    rng = np.random.default_rng(13)
    cells = sorted(int(c) for t in range(3) for c in rng.choice(np.flatnonzero(b.type_of_cell == t), 5, replace=False))
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM, cells=cells)


# FP64 form: rounding of the per-cell sums (6.8e-15 measured on B300 over 10^4 and 2*10^4
# cells).  FP32 form: the gradient's FP32 rounding leaves its vertex sum off zero by about
# 6e-8 of |g| times sqrt(n), and the velocities are stored in FP32 (1.3e-6 measured).
MOMENTUM_BAR = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("workload", ["mixed10k", "stress20k"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_momentum_balance_every_cell(workload, prec):
    """Every cell of the full-size mixed workloads in the default launch configuration, not a
    sample: over one step each cell's momentum sum_i m_i v_i changes by dt sum_i f_i, the
    balance the step keeps at any iteration count (pinned on the oracle's step).  Error per
    cell = max over components of the imbalance / sum_i m_i |v_i^{n+1}|_inf; masses from the
    oracle's rest state of each type."""
    nat = _native()
    b = (I.heterogeneous_batch(4500, 4500, 1000, seed=1002) if workload == "mixed10k"
         else I.stress_mix_batch())
    precision = nat.FP64 if prec == "fp64" else nat.FP32FORM
    x, v, f = b.x, b.v, b.f
    if prec == "fp32":
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    _, vg, _, st, _ = Runner(b, precision).step(x, v, f, iters=b.iters)
    assert np.all(st == O.STATUS_OK)
    masses = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt).rest.mass for t in b.types]
    m = np.concatenate([masses[t] for t in b.type_of_cell])
    starts = np.asarray(b.offsets[:-1], dtype=np.int64)
    p_new = np.add.reduceat(m * vg, starts, axis=1)
    p_expect = np.add.reduceat(m * v, starts, axis=1) + b.dt * np.add.reduceat(f, starts, axis=1)
    scale = np.add.reduceat(m * np.max(np.abs(vg), axis=0), starts)
    err = np.max(np.abs(p_new - p_expect), axis=0) / scale
    print(f"{workload} {prec}: max momentum imbalance {err.max():.3e} over {b.ncells} cells")
    assert err.max() <= MOMENTUM_BAR[prec]


@pytest.mark.parametrize("width", [None, 0])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_collapsed_cells_are_flagged_and_stay(prec, width):
    """A strain-only type (bending, area and volume weights 0) with two of its three cells
    collapsed to a point: every triangle of those is degenerate and the gradient exactly
    zero, so they keep their state exactly, report residual 0 and only the degenerate
    status, as the oracle's step does; the ordinary cell between them matches the oracle.
    CTA iteration kernels (default width) and the one-warp kernels (width 0)."""
    nat = _native()
    mesh = I.rbc_mesh(2)
    spec = I.CellTypeSpec(mesh, I.Material(1.0, 0.0, 0.0, 0.0, 1.1))
    p0, p2 = np.array([2.0, -1.0, 0.5]), np.array([-4.0, 8.0, 0.25])      # exact in FP32
    xs = [np.tile(p0, (mesh.n, 1)), mesh.verts + np.array([20.0, 0.0, 0.0]), np.tile(p2, (mesh.n, 1))]
    z = [np.zeros_like(xs[0])] * 3
    f = [np.zeros_like(xs[0]), I.stretch_forces(mesh.verts, rng=np.random.default_rng(3)), np.zeros_like(xs[0])]
    b = I._assemble([spec], [0, 0, 0], xs, z, f, [4, 4, 4], I.DT_DEFAULT, 0)
    precision = nat.FP64 if prec == "fp64" else nat.FP32FORM
    x, v, fv = b.x, b.v, b.f
    if prec == "fp32":
        x, v, fv = (a.astype(np.float32).astype(np.float64) for a in (x, v, fv))
    r = Runner(b, precision)
    if width is not None:
        r.batch.set_iter_width(0, width)
    xg, vg, res, st, _ = r.step(x, v, fv, iters=b.iters)
    ref = O.batch_step(oracle_types(b), b.type_of_cell, b.offsets, x, v, fv, b.iters)
    for c in (0, 2):
        s_ = b.cell_slice(c)
        assert ref["status"][c] == O.STATUS_DEGENERATE and ref["residual"][c] == 0.0
        assert st[c] == nat.CELL_DEGENERATE
        assert res[c] == 0.0
        assert np.array_equal(xg[:, s_], x[:, s_])
        assert np.array_equal(vg[:, s_], np.zeros_like(vg[:, s_]))
    assert st[1] == ref["status"][1] == O.STATUS_OK
    bar = FP64_BAR if prec == "fp64" else FP32_BAR
    s1 = b.cell_slice(1)                      # (the collapsed cells have no radius to divide by)
    xr = ref["x"][:, s1]
    rad = np.max(np.linalg.norm(xr - xr.mean(axis=1, keepdims=True), axis=0))
    assert np.max(np.abs(xg[:, s1] - xr)) / rad <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_largest_size_class_parity(prec):
    """Two placed 10242-vertex RBCs (icosphere subdivision 5; factor nnz 0.86 M), one step
    against the oracle: the largest cells the tests step (type setup grows to about a minute
    at 40962 vertices).  Their solve vectors exceed shared memory (workspace placement) and
    their iteration arrays exceed a CTA's shared memory (one-warp iteration kernels)."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=2, seed=1001, subdiv=5)
    assert b.types[0].mesh.n == 10242
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_counts_beyond_the_split_bound_run_fused(prec):
    """Per-cell counts above the split kernels' bound of 32 iterations (40 and 33, beside
    ordinary counts) send the step to the fused kernel; every cell matches the oracle."""
    nat = _native()
    b = I.small_mixed_batch()
    it = b.iters.copy()
    it[0], it[4] = 40, 33
    compare(b, nat.FP64 if prec == "fp64" else nat.FP32FORM, iters=it)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_counts_above_max_iters_stop_there_with_the_limit_status(prec):
    """Split mode with a caller-given max_iters of 3: cells whose count is above it run 3
    iterations and report NPFEM_CELL_ITER_LIMIT alone; they equal the oracle's 3-iteration
    step, and the other cells their own counts' steps."""
    nat = _native()
    b = I.small_mixed_batch()
    it = b.iters.copy()
    it[1], it[2], it[5] = 6, 3, 1
    precision = nat.FP64 if prec == "fp64" else nat.FP32FORM
    x, v, f = b.x, b.v, b.f
    if prec == "fp32":
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    xg, vg, res, st, _ = Runner(b, precision).step(x, v, f, iters=it, max_iters=3)
    capped = np.minimum(it, 3)
    ref = O.batch_step(oracle_types(b), b.type_of_cell, b.offsets, x, v, f, capped)
    assert np.array_equal(st, np.where(it > 3, nat.CELL_ITER_LIMIT, O.STATUS_OK))
    assert np.all(ref["status"] == O.STATUS_OK)
    bar = FP64_BAR if prec == "fp64" else FP32_BAR
    assert cell_errors(b, xg, ref["x"]).max() <= bar
    assert cell_errors(b, vg * b.dt, ref["v"] * b.dt, radius_from=ref["x"]).max() <= bar


def test_uncoloured_type_runs_the_warp_kernels():
    """A type whose mesh would need more than 64 colour classes (a 70-gon bipyramid, 70
    triangles at each pole) has no CTA iteration kernels: its width is 0, setting one is
    refused, and its cells (FP32 form, beside a coloured RBC type on the CTA kernels) match
    the oracle."""
    nat = _native()
    types = [I.CellTypeSpec(I.bipyramid(70), I.RBC_MATERIAL), I.CellTypeSpec(I.rbc_mesh(2), I.RBC_MATERIAL)]
    b = I.placed_cells(types, [0, 1, 0, 1, 0], 1012, 4)
    r = Runner(b, nat.FP32FORM)
    assert r.batch.get_iter_width(0) == (0, 0) and r.batch.get_iter_width(1)[0] == 2   # 162 vertices
    with pytest.raises(nat.NpfemError):
        r.batch.set_iter_width(0, 4)
    compare(b, nat.FP32FORM, steps=2)
    compare(b, nat.FP64)


def test_heterogeneous_types_and_iterations():
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=6, n_rbc4=3, n_plt=5, seed=1002)
    compare(b, nat.FP64)
    compare(b, nat.FP32FORM)


def test_zero_iterations_returns_prediction():
    nat = _native()
    b = I.small_mixed_batch()
    iters = np.zeros(b.ncells, np.int32)
    r = Runner(b, nat.FP64)
    xg, vg, res, st, _ = r.step(b.x, b.v, b.f, iters=iters)
    mass = [O.rest_state(t.mesh.verts, t.mesh.tris, *t.material.as_tuple(), b.dt).mass for t in b.types]
    for c in range(b.ncells):
        s = b.cell_slice(c)
        m = mass[b.type_of_cell[c]]
        y = b.x[:, s] + b.dt * b.v[:, s] + b.dt ** 2 * b.f[:, s] / m[None, :]
        assert np.allclose(xg[:, s], y, rtol=0, atol=1e-12)
        assert res[c] == 1.0 or np.isclose(res[c], 1.0)


def test_rest_state_stays_at_rest():
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=8, seed=3)
    for prec in (nat.FP64, nat.FP32FORM):
        r = Runner(b, prec)
        x = b.x if prec == nat.FP64 else b.x.astype(np.float32).astype(np.float64)
        xg, vg, res, st, _ = r.step(x, np.zeros_like(x), np.zeros_like(x))
        tol = 1e-12 if prec == nat.FP64 else 2e-5
        assert np.max(np.abs(xg - x)) <= tol * 200
        assert np.all(st == 0)


def test_nonfinite_force_sets_status_only_for_that_cell():
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=6, seed=4)
    f = b.f.copy()
    s = b.cell_slice(2)
    f[0, s.start + 5] = np.nan
    r = Runner(b, nat.FP64)
    xg, vg, res, st, _ = r.step(b.x, b.v, f)
    assert st[2] & nat.CELL_NONFINITE
    assert all(st[c] == 0 for c in range(6) if c != 2)
    assert np.all(np.isfinite(xg[:, b.cell_slice(0)]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["homogeneous", "mixed"])
def test_host_buffer_step_matches_device_step(prec, kind):
    """npfem_step_host (chunks of cells copied in, stepped and copied out in a pipeline;
    in the mixed batch the chunk boundaries cut through every type's cell list) gives the
    device-buffer step's results bit for bit, from pinned and from pageable host arrays."""
    nat = _native()
    b = (I.homogeneous_rbc_batch(ncells=10, seed=6) if kind == "homogeneous"
         else I.heterogeneous_batch(n_rbc3=7, n_rbc4=3, n_plt=6, seed=1010))
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    r = Runner(b, p)
    xg, vg, res, st, _ = r.step(b.x, b.v, b.f, iters=b.iters)
    npdt = np.float64 if prec == "fp64" else np.float32
    for pinned in (False, True):
        if pinned:
            xh, vh, fh = (torch.tensor(a, dtype=torch.float64 if prec == "fp64" else torch.float32).pin_memory().numpy()
                          for a in (b.x, b.v, b.f))
        else:
            xh, vh, fh = (np.array(a, dtype=npdt, copy=True) for a in (b.x, b.v, b.f))
        rh = np.zeros(b.ncells)
        sh = np.zeros(b.ncells, np.int32)
        r.batch.step_host(xh, vh, fh, iters=np.ascontiguousarray(b.iters), residual=rh, status=sh)
        assert np.array_equal(xh.astype(np.float64), xg) and np.array_equal(vh.astype(np.float64), vg)
        assert np.array_equal(rh, res) and np.array_equal(sh, st)


def test_empty_batch_is_a_no_op():
    nat = _native()
    t = nat.CellType(I.icosahedron().verts, I.icosahedron().tris, I.RBC_MATERIAL.as_tuple(), 0.1)
    bt = nat.Batch([t], np.zeros(0, np.int32), nat.FP64)
    x = torch.zeros(3, 0, dtype=torch.float64, device="cuda")
    bt.step(x, x.clone(), x.clone())
    torch.cuda.synchronize()


def test_rollout_tracks_oracle():
    """20 steps of the single RBC on both sides from the same start (informational bar)."""
    nat = _native()
    b = I.single_rbc()
    r = Runner(b, nat.FP64)
    ots = oracle_types(b)
    x, v = b.x.copy(), b.v.copy()
    xo, vo = b.x.copy(), b.v.copy()
    for s in range(20):
        x, v, *_ = r.step(x, v, b.f, iters=b.iters)
        ref = O.batch_step(ots, b.type_of_cell, b.offsets, xo, vo, b.f, b.iters)
        xo, vo = ref["x"], ref["v"]
    assert cell_errors(b, x, xo).max() < 1e-8


@pytest.mark.parametrize("width", [None, 0])
def test_phase_cycle_telemetry(width):
    """Per-phase cycle counters are off by default (a step adds nothing), and once
    switched on accumulate over steps and reset on request; for the CTA iteration
    kernels (default width) and the one-warp kernels (width 0), with bit-identical
    states whether counting or not."""
    nat = _native()
    b = I.homogeneous_rbc_batch(ncells=8, seed=11)
    r = Runner(b, nat.FP32FORM)
    if width is not None:
        r.batch.set_iter_width(0, width)
    r.batch.phase_cycles(reset=True)
    plain = r.step(b.x, b.v, b.f)
    assert all(v == 0 for v in r.batch.phase_cycles().values())
    r.batch.set_phase_counting(True)
    counted = r.step(b.x, b.v, b.f)
    for a, c_ in zip(plain, counted):
        assert np.array_equal(a, c_)
    c = r.batch.phase_cycles(reset=True)
    assert c["solve"] > 0 and c["objective"] > 0 and c["two_loop"] > 0 and c["write"] > 0
    assert c["gather"] < c["objective"] and c["area_volume"] < c["objective"]
    assert all(v == 0 for v in r.batch.phase_cycles().values())


def test_launch_shapes_give_identical_results():
    """A cell's arithmetic does not depend on the launch shape: every feasible shape
    (warps per CTA, CTAs per SM, solve vector in shared memory or workspace) gives
    bit-identical states; the autotuner keeps one of them."""
    nat = _native()
    from paper_2011_04332_b300 import tuning
    b = I.heterogeneous_batch(n_rbc3=9, n_rbc4=2, n_plt=7, seed=1002)
    r = Runner(b, nat.FP32FORM)
    x0, v0, *_ = r.step(b.x, b.v, b.f, iters=b.iters)
    for t in range(len(b.types)):
        n = b.types[t].mesh.n
        shapes = tuning.candidate_shapes(n)
        for shape in shapes[:5] + [sh for sh in shapes if sh[3] == 1][:3] + [(3, 1, 1, 0)]:
            r.batch.set_launch(t, *shape)
            assert r.batch.get_launch(t)["warps_per_block"] == shape[0]
            x1, v1, *_ = r.step(b.x, b.v, b.f, iters=b.iters)
            assert np.array_equal(x1, x0) and np.array_equal(v1, v0), (t, shape)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    res = tuning.autotune(r.batch, T(b.x), T(b.v), T(b.f), iters=torch.tensor(b.iters, device=dev))
    assert set(res) == {0, 1, 2}
    x2, v2, *_ = r.step(b.x, b.v, b.f, iters=b.iters)
    assert np.array_equal(x2, x0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_mode_launch_shapes_give_identical_results(prec):
    """The fused persistent kernel (mode 0) under the launch shapes of
    npfem_batch_set_launch, the per-coordinate choice with the solve vector in the
    workspace included (which then sweeps the whole vector): identical states."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=5, n_rbc4=2, n_plt=5, seed=1013)
    r = Runner(b, nat.FP64 if prec == "fp64" else nat.FP32FORM)
    r.batch.set_mode(False)
    ref = r.step(b.x, b.v, b.f, iters=b.iters)
    for shape in ((4, 3, False, False), (2, 2, False, True), (1, 8, True, False), (3, 1, True, True)):
        for t in range(len(b.types)):
            n = b.types[t].mesh.n
            if shape[2] and shape[0] * (8 if shape[3] else 24) * (n + 1) > 72 * 1024:
                continue  # vectors that do not fit shared memory at this width
            r.batch.set_launch(t, *shape)
        out = r.step(b.x, b.v, b.f, iters=b.iters)
        for a, c in zip(ref, out):
            assert np.array_equal(a, c), shape
    r.batch.set_mode(True)


def test_cuda_graph_replay_equals_direct_steps():
    """npfem_step is capturable: a captured step replayed twice gives the same state as
    two direct calls."""
    nat = _native()
    b = I.small_mixed_batch(seed=21)
    r = Runner(b, nat.FP32FORM)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    it = torch.tensor(b.iters, device=dev)
    xa, va, f = T(b.x), T(b.v), T(b.f)
    for _ in range(2):
        r.batch.step(xa, va, f, iters=it)
    xb, vb = T(b.x), T(b.v)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            r.batch.step(xb, vb, f, iters=it)
    torch.cuda.current_stream().wait_stream(s)
    xb.copy_(T(b.x))
    vb.copy_(T(b.v))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(va, vb)


def test_kernel_timing_eager_and_in_graph():
    """Per-kernel CUDA-event timing of split-mode steps: one k_begin and, per iteration up
    to the batch's largest count, one k_solve and one k_iter per cell type, with positive
    durations, both for direct steps and for replays of a captured step; the timed step
    is unchanged by the events."""
    nat = _native()
    b = I.small_mixed_batch(seed=23)
    r = Runner(b, nat.FP32FORM)
    dev = torch.device("cuda:0")
    T = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    it = torch.tensor(b.iters, device=dev)
    kmax = int(b.iters.max())
    present = sorted({int(t) for t in b.type_of_cell})
    xa, va, f = T(b.x), T(b.v), T(b.f)
    r.batch.step(xa, va, f, iters=it)
    with pytest.raises(nat.NpfemError):
        r.batch.kernel_times(present[0])
    r.batch.set_kernel_timing(True)
    xb, vb = T(b.x), T(b.v)
    r.batch.step(xb, vb, f, iters=it)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    for t in present:
        kt = r.batch.kernel_times(t)
        assert [kt[k][1] for k in nat.Batch.KERNELS] == [1, kmax, kmax]
        assert all(kt[k][0] > 0 for k in nat.Batch.KERNELS)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    xc, vc = T(b.x), T(b.v)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            r.batch.step(xc, vc, f, iters=it)
    torch.cuda.current_stream().wait_stream(s)
    xc.copy_(T(b.x))
    vc.copy_(T(b.v))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(xa, xc) and torch.equal(va, vc)
    for t in present:
        kt = r.batch.kernel_times(t)
        assert [kt[k][1] for k in nat.Batch.KERNELS] == [1, kmax, kmax]
        assert all(kt[k][0] > 0 for k in nat.Batch.KERNELS)
        sp = r.batch.kernel_spans(t)
        # event times resolve to about half a microsecond
        assert all(0 < sp[k] <= kt[k][0] + 0.01 for k in nat.Batch.KERNELS)
    spall = r.batch.kernel_spans(-1)
    assert all(spall[k] >= max(r.batch.kernel_spans(t)[k] for t in present) - 0.01 for k in nat.Batch.KERNELS)
    r.batch.set_kernel_timing(False)


def _assert_modes_agree(fused, split, prec, b):
    """The fused and the split kernels are compiled separately, and the compiler may
    contract multiply-adds differently in them, so their results agree to rounding of a
    few iterations: 1e-12 (FP64) or 1e-6 (FP32 form) of the cell radius plus four ulps
    of the stored coordinates; statuses exactly."""
    xf, vf, rf, sf, af = fused
    xs, vs, rs, ss, as_ = split
    assert np.array_equal(sf, ss)
    rel, dt_ = (1e-12, np.float64) if prec == "fp64" else (1e-6, np.float32)
    for c in range(b.ncells):
        s = b.cell_slice(c)
        rad = np.max(np.linalg.norm(xf[:, s] - xf[:, s].mean(axis=1, keepdims=True), axis=0))
        ulp = float(np.spacing(dt_(np.max(np.abs(xf[:, s])))))
        assert np.max(np.abs(xf[:, s] - xs[:, s])) <= rel * rad + 4 * ulp
        assert np.max(np.abs(vf[:, s] - vs[:, s])) * b.dt <= rel * rad + 4 * ulp
    assert np.allclose(rf, rs, rtol=1e-3 if prec != "fp64" else 1e-8, atol=1e-7 if prec != "fp64" else 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_split_and_fused_modes_agree(prec):
    """The split kernels (k_begin, k_solve, k_iter) and the fused persistent kernel run the
    same arithmetic, with ragged per-cell iteration counts including zero; split launch
    shapes do not change the split results at all."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=7, n_rbc4=3, n_plt=6, seed=1005)
    it = b.iters.copy()
    it[0] = 0
    it[3] = 1
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    r = Runner(b, p)
    r.batch.set_mode(False)
    fused = r.step(b.x, b.v, b.f, iters=it)
    r.batch.set_mode(True)
    assert r.batch.get_split_launch(0)[1] is True
    split = r.step(b.x, b.v, b.f, iters=it)
    _assert_modes_agree(fused, split, prec, b)
    # one-warp solves (placements 0 and 1) in two different shapes: identical results
    for t, shape in enumerate([(2, 8, 2, 7, 1, 0), (2, 8, 2, 8, 0, 0), (4, 4, 2, 7, 1, 0)]):
        r.batch.set_split_launch(t, shape)
    split1 = r.step(b.x, b.v, b.f, iters=it)
    _assert_modes_agree(fused, split1, prec, b)
    for t, shape in enumerate([(4, 3, 1, 14, 1, 1), (2, 3, 3, 1, 0, 0), (4, 2, 2, 2, 0, 1)]):
        r.batch.set_split_launch(t, shape)
    split2 = r.step(b.x, b.v, b.f, iters=it)
    for a, c in zip(split1, split2):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("cells", [2, 3, 4])
def test_multi_cell_solve_is_identical(prec, cells):
    """Several cells per solve warp (shared factor, 3 x cells right-hand sides per entry)
    in every vector placement gives the one-cell split results bit for bit (and the fused
    kernel's, as above), with ragged iteration counts (short last groups, cells dropping
    out of the active lists)."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=9, n_rbc4=3, n_plt=11, seed=1006)
    it = b.iters.copy()
    it[0] = 0
    it[5] = 1
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    r = Runner(b, p)
    r.batch.set_mode(False)
    fused = r.step(b.x, b.v, b.f, iters=it)
    r.batch.set_mode(True)
    for t in range(len(b.types)):            # one cell per warp, vectors in shared memory
        r.batch.set_split_launch(t, (2, 4, 1, 2, 1, 0, 1))
    one = r.step(b.x, b.v, b.f, iters=it)
    _assert_modes_agree(fused, one, prec, b)
    for placement in [(1, 0), (1, 1), (0, 0)]:
        for t, wpb in ((0, 1), (1, 2), (2, 1)):
            shape = (2, 4, wpb, 2, placement[0], placement[1], cells)
            try:
                r.batch.set_split_launch(t, shape)
            except nat.NpfemError:          # vectors of 2562-vertex cells exceed shared memory
                r.batch.set_split_launch(t, (2, 4, wpb, 2, 0, 0, cells))
            assert r.batch.get_split_launch(t)[0][6] == cells
        split = r.step(b.x, b.v, b.f, iters=it)
        for a, c in zip(one, split):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("warps,cells", [(2, 1), (4, 1), (6, 1), (8, 1), (2, 2), (4, 2)])
def test_cta_cooperative_solve(prec, warps, cells):
    """Placement 2: the warps of a CTA sweep one cell's (or two cells') shared solve
    vectors through the level packing of the factor, for every type of a mixed batch
    (162, 642 and 2562 vertices, 3..8 iterations, so the lists of cells still iterating
    have odd lengths): parity with the oracle at the usual bars over two steps, agreement
    with the one-warp solve to rounding (the level packing applies the same updates in
    another order), and two cells per CTA give the one-cell CTA's results bit for bit."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=6, n_rbc4=4, n_plt=5, seed=1007)
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    shapes = {t: (2, 4, warps, 2, 2, 0, cells) for t in range(len(b.types))}
    compare(b, p, steps=2, shapes=shapes)
    r = Runner(b, p)
    for t in range(len(b.types)):            # one cell per warp, vectors in shared memory
        r.batch.set_split_launch(t, (2, 4, 1, 2, 1, 0, 1))
    one = r.step(b.x, b.v, b.f, iters=b.iters)
    for t, shape in shapes.items():
        r.batch.set_split_launch(t, shape)
        assert r.batch.get_split_launch(t)[0] == shape
    cta = r.step(b.x, b.v, b.f, iters=b.iters)
    _assert_modes_agree(one, cta, prec, b)
    if cells == 2:
        for t in range(len(b.types)):
            r.batch.set_split_launch(t, (2, 4, warps, 2, 2, 0, 1))
        single = r.step(b.x, b.v, b.f, iters=b.iters)
        for a, c in zip(single, cta):
            assert np.array_equal(a, c)


def test_cta_cooperative_shape_validation():
    """Placement 2 takes 2, 4, 6 or 8 warps per CTA and one cell, or 2 or 4 warps and
    two cells, interleaved coordinates."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=2, n_rbc4=1, n_plt=1, seed=1008)
    r = Runner(b, nat.FP64)
    for bad in [(2, 4, 3, 2, 2, 0, 1), (2, 4, 2, 2, 2, 1, 1), (2, 4, 4, 2, 2, 0, 3), (2, 4, 6, 2, 2, 0, 2),
                (2, 4, 2, 2, 3, 0, 1), (2, 4, 5, 2, 2, 0, 1), (2, 4, 6, 2, 1, 0, 1)]:
        with pytest.raises(nat.NpfemError):
            r.batch.set_split_launch(0, bad)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_groups_leave_results_unchanged(prec):
    """Cells of a type split into 2..4 phase-offset chains (their solves take turns, their
    iteration kernels overlap the other groups' solves) give the one-group results bit
    for bit, with the solves on high-priority streams of their own or not, directly and
    replayed from a captured CUDA graph; groups outside 1..4 are rejected."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=9, n_rbc4=3, n_plt=7, seed=1009)
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    r = Runner(b, p)
    ref = r.step(b.x, b.v, b.f, iters=b.iters)
    for groups in (2, 3, 4):
        for t in range(len(b.types)):
            r.batch.set_groups(t, groups)
            assert r.batch.get_groups(t) == groups
        out = r.step(b.x, b.v, b.f, iters=b.iters)
        for a, c in zip(ref, out):
            assert np.array_equal(a, c)
        # the chains' solves on streams of their own (default) or on the chains' streams
        r.batch.set_solve_streams(False)
        out = r.step(b.x, b.v, b.f, iters=b.iters)
        r.batch.set_solve_streams(True)
        for a, c in zip(ref, out):
            assert np.array_equal(a, c)
    dev = torch.device("cuda:0")
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    T = lambda a: torch.tensor(a, dtype=dt_, device=dev)
    it = torch.tensor(b.iters, device=dev)
    xg, vg, f = T(b.x), T(b.v), T(b.f)
    r.batch.step(xg, vg, f, iters=it)        # warm-up (reads the iteration bound once)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            r.batch.step(xg, vg, f, iters=it)
    torch.cuda.current_stream().wait_stream(s)
    xg.copy_(T(b.x))
    vg.copy_(T(b.v))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(xg.double().cpu().numpy(), ref[0]) and np.array_equal(vg.double().cpu().numpy(), ref[1])
    for bad in (0, 5):
        with pytest.raises(nat.NpfemError):
            r.batch.set_groups(0, bad)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_iteration_kernel_widths(prec):
    """Split-mode iteration kernels with one CTA per cell (positions, trial displacement and
    gradient in shared memory, elements by colour class) at widths 1 to 16 warps, and the
    one-warp-per-cell kernels (width 0): every width matches the oracle at the usual bars
    over two steps with ragged iteration counts (zero and one included), the widths agree
    with each other to rounding (the width sets the order of a cell's sums), and a width
    keeps its bits under other iteration launch shapes."""
    nat = _native()
    b = I.heterogeneous_batch(n_rbc3=5, n_rbc4=2, n_plt=4, seed=1011)
    it = b.iters.copy()
    it[0] = 0
    it[2] = 1
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    r = Runner(b, p)
    defaults = [r.batch.get_iter_width(t)[0] for t in range(len(b.types))]
    assert defaults == ([0] * len(b.types) if prec == "fp64" else [4, 8, 2])
    ref = r.step(b.x, b.v, b.f, iters=it)
    for w in (0, 1, 2, 4, 8, 16):
        for t in range(len(b.types)):
            r.batch.set_iter_width(t, w)
            assert r.batch.get_iter_width(t)[0] == w
            assert (r.batch.get_iter_width(t)[1] > 0) == (w > 0)
        out = r.step(b.x, b.v, b.f, iters=it)
        _assert_modes_agree(ref, out, prec, b)
        shapes = {t: (2, 8) + tuple(r.batch.get_split_launch(t)[0][2:]) for t in range(len(b.types))}
        compare(b, p, steps=2, iters=it, width=w)
        for t, sh in shapes.items():
            r.batch.set_split_launch(t, (4, 3) + sh[2:])
        again = r.step(b.x, b.v, b.f, iters=it)
        for a, c in zip(out, again):
            assert np.array_equal(a, c), w
        for t, sh in shapes.items():
            r.batch.set_split_launch(t, sh)
    for bad in (-1, 3, 6, 17, 32):
        with pytest.raises(nat.NpfemError):
            r.batch.set_iter_width(0, bad)
