"""GPU parity of collisions: contact detection (integer decisions bit for bit, planes to
FP64 rounding) and the step with contact penalties against the oracle, plus the
execution variants (split / fused, graph replay, host buffers) and argument errors.

The detection compares FP64 squared distances evaluated in the same order on both
sides, so the matched vertices and cells must be identical; in the FP32 form both
sides see the same FP32-rounded positions."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_BAR = 1e-10
FP32_BAR = 1e-5
RADIUS, DELTA, WEIGHT = 0.6, 0.1, 40.0


def _native():
    from paper_2011_04332_b300 import native
    return native


def _small_packing(seed=3):
    """8 RBCs (162 vertices) and 4 platelets (42 vertices) at 35 % volume fraction."""
    return I.packing_batch(8, 4, hematocrit=0.35, seed=seed, rbc_subdiv=2, plt_subdiv=1, iters=4)


def _setup(b, prec, collisions=True, radius=RADIUS):
    nat = _native()
    types = [nat.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    batch = nat.Batch(types, b.type_of_cell, prec)
    if collisions:
        batch.set_collisions(radius, DELTA, WEIGHT)
    return types, batch


def _inputs(b, prec):
    nat = _native()
    x, v, f = b.x.copy(), b.v.copy(), b.f.copy()
    if prec == nat.FP32FORM:
        x, v, f = (a.astype(np.float32).astype(np.float64) for a in (x, v, f))
    return x, v, f


def _step(batch, prec, x, v, f, iters, graph=False):
    nat = _native()
    dev = torch.device("cuda:0")
    dt = torch.float64 if prec == nat.FP64 else torch.float32
    X = torch.tensor(x, dtype=dt, device=dev)
    V = torch.tensor(v, dtype=dt, device=dev)
    F = torch.tensor(f, dtype=dt, device=dev)
    it = torch.tensor(np.asarray(iters, np.int32), device=dev)
    nc, N = batch.ncells, batch.n_total
    res = torch.zeros(nc, dtype=torch.float64, device=dev)
    st = torch.zeros(nc, dtype=torch.int32, device=dev)
    al = torch.zeros((nc, 8), dtype=torch.float64, device=dev)
    if graph:
        X0, V0 = X.clone(), V.clone()
        batch.step(X, V, F, iters=it, residual=res, status=st, alpha_log=al)   # warm-up outside capture
        torch.cuda.synchronize()
        X.copy_(X0)
        V.copy_(V0)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                batch.step(X, V, F, iters=it, residual=res, status=st, alpha_log=al)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        X.copy_(X0)
        V.copy_(V0)
        g.replay()
    else:
        batch.step(X, V, F, iters=it, residual=res, status=st, alpha_log=al)
    cnt = torch.zeros(N, dtype=torch.int32, device=dev)
    vert = torch.zeros((N, 2), dtype=torch.int32, device=dev)
    plane = torch.zeros((N, 2, 4), dtype=torch.float64, device=dev)
    if batch.collisions_on:
        batch.contacts(cnt, vert, plane)
    torch.cuda.synchronize()
    return {"x": X.double().cpu().numpy(), "v": V.double().cpu().numpy(), "residual": res.cpu().numpy(),
            "status": st.cpu().numpy(), "alpha": al.cpu().numpy(), "count": cnt.cpu().numpy(),
            "vertex": vert.cpu().numpy(), "plane": plane.cpu().numpy()}


def _check_contacts(b, got, ref_con, x, vertices=None):
    """Integer decisions identical; normals and plane offsets to FP64 rounding.  The
    GPU offset is relative to the first vertex of vertex i's cell."""
    sel = np.arange(b.n_total) if vertices is None else np.asarray(vertices)
    assert np.array_equal(got["count"][sel], ref_con["count"][sel])
    vref = np.where(ref_con["vertex"] >= 0, ref_con["vertex"], -1)
    assert np.array_equal(got["vertex"][sel], vref[sel])
    cell_of = np.repeat(np.arange(b.ncells), np.diff(b.offsets))
    for i in sel:
        for k in range(int(ref_con["count"][i])):
            assert np.allclose(got["plane"][i, k, :3], ref_con["normal"][i, k], rtol=0, atol=1e-13)
            anchor = x[:, b.offsets[cell_of[i]]]
            c_rel = ref_con["offset"][i, k] - float(ref_con["normal"][i, k] @ anchor)
            assert got["plane"][i, k, 3] == pytest.approx(c_rel, rel=0, abs=1e-11)
    return int(np.sum(got["count"][sel]))


def _check_state(b, prec, got, ref, cells, ots):
    nat = _native()
    bar = FP64_BAR if prec == nat.FP64 else FP32_BAR
    for c in cells:
        s = b.cell_slice(c)
        xr = ref["x"][:, s]
        rad = np.max(np.linalg.norm(xr - xr.mean(axis=1, keepdims=True), axis=0))
        assert np.max(np.abs(got["x"][:, s] - xr)) / rad <= bar, c
        assert np.max(np.abs(got["v"][:, s] - ref["v"][:, s])) * b.dt / rad <= bar, c
        assert got["status"][c] == ref["status"][c]
        g = np.asarray(ref["grad_norms"][c])
        # a cell at rest with neither force nor contact has a gradient at the rounding
        # level of its positions (inertial scale m/dt^2 x radius): its line-search
        # decisions compare rounding noise, and only its state is checked
        scale = float(np.max(ots[int(b.type_of_cell[c])].rest.mass)) / b.dt ** 2 * rad
        if prec == nat.FP64 and g[0] > 1e-9 * scale:
            k = min(int(b.iters[c]), 8)
            assert np.array_equal(got["alpha"][c, :k], np.array(ref["alphas"][c][:k])), (c, g / g[0])


@pytest.mark.parametrize("mode", ["split", "fused"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_contacts_and_step_parity(mode, prec):
    """Small packing batch (mixed types, overlapping at 35 % volume fraction), two
    consecutive steps, each from the oracle's previous state with fresh detection."""
    nat = _native()
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = _small_packing()
    _, batch = _setup(b, p)
    batch.set_mode(mode == "split")
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    x, v, f = _inputs(b, p)
    for s in range(2):
        got = _step(batch, p, x, v, f, b.iters)
        ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, b.iters, collisions=(RADIUS, DELTA, WEIGHT))
        assert _check_contacts(b, got, ref["contacts"], x) > 100
        _check_state(b, p, got, ref, range(b.ncells), ots)
        x, v = ref["x"], ref["v"]
        if p == nat.FP32FORM:
            x, v = (a.astype(np.float32).astype(np.float64) for a in (x, v))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_contacts_with_large_cells(prec):
    """3 RBCs of 2562 vertices (5120 triangles: the normals kernel keeps 123 KB of
    triangle normals in shared memory) and 3 platelets of 162 vertices, overlapping at
    35 % volume fraction: contacts and step against the oracle."""
    nat = _native()
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = I.packing_batch(3, 3, hematocrit=0.35, seed=21, rbc_subdiv=4, plt_subdiv=2, iters=3)
    _, batch = _setup(b, p)
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    x, v, f = _inputs(b, p)
    got = _step(batch, p, x, v, f, b.iters)
    ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, b.iters, collisions=(RADIUS, DELTA, WEIGHT))
    assert _check_contacts(b, got, ref["contacts"], x) > 100
    _check_state(b, p, got, ref, range(b.ncells), ots)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_contact_free_collisions_equal_plain_step(prec):
    """Collisions on but no vertex within the radius of another cell: the step is bit
    for bit the step without collisions (an empty contact pass adds exact zeros)."""
    nat = _native()
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = I.homogeneous_rbc_batch(ncells=24, seed=1001, velocity_sigma=0.02)
    x, v, f = _inputs(b, p)
    _, plain = _setup(b, p, collisions=False)
    _, coll = _setup(b, p, radius=1e-3)
    r0 = _step(plain, p, x, v, f, b.iters)
    r1 = _step(coll, p, x, v, f, b.iters)
    assert np.sum(r1["count"]) == 0
    for k in ("x", "v", "residual", "status", "alpha"):
        assert np.array_equal(r0[k], r1[k]), k
    coll.set_collisions(None)
    r2 = _step(coll, p, x, v, f, b.iters)
    assert np.array_equal(r0["x"], r2["x"])


def test_graph_replay_and_host_buffers_with_collisions():
    """CUDA-graph replay of a step with collisions equals the direct call bit for bit,
    and so does npfem_step_host."""
    nat = _native()
    b = _small_packing(seed=9)
    _, batch = _setup(b, nat.FP64)
    x, v, f = _inputs(b, nat.FP64)
    direct = _step(batch, nat.FP64, x, v, f, b.iters)
    replay = _step(batch, nat.FP64, x, v, f, b.iters, graph=True)
    for k in ("x", "v", "residual", "status", "count", "vertex", "plane"):
        assert np.array_equal(direct[k], replay[k]), k
    hx, hv, hf = (np.array(a, copy=True) for a in (x, v, f))
    res = np.zeros(b.ncells)
    st = np.zeros(b.ncells, np.int32)
    batch.step_host(hx, hv, hf, iters=b.iters, residual=res, status=st)
    assert np.array_equal(hx, direct["x"]) and np.array_equal(hv, direct["v"])
    assert np.array_equal(res, direct["residual"])


def _penetrations(b, got, x):
    """Matches whose gap at the step's input is negative (vertex inside the other
    cell's tangent plane): their number and their summed depth."""
    cell_of = np.repeat(np.arange(b.ncells), np.diff(b.offsets))
    anchors = x[:, b.offsets[:-1]][:, cell_of]
    n, depth = 0, 0.0
    for k in range(2):
        used = got["count"] > k
        gap = np.einsum("dn,nd->n", x - anchors, got["plane"][:, k, :3]) - got["plane"][:, k, 3]
        inside = used & (gap < 0)
        n += int(np.sum(inside))
        depth += float(-np.sum(gap[inside]))
    return n, depth


def test_packing_pushes_cells_apart():
    """Packing: 64 RBCs (642 vertices) placed at random at 35 % volume fraction, FP32
    form, 30 steps with collisions (velocities carried).  The first steps cut the number
    and the summed depth of penetrating matches, and every state stays finite (a
    strongly pushed triangle may report DEGENERATE).  Resolving every overlap takes
    far more steps: vertices deeper than the search radius are not matched until the
    surface around them has moved."""
    nat = _native()
    b = I.packing_batch(64, 0, hematocrit=0.35, seed=12)
    _, batch = _setup(b, nat.FP32FORM, radius=0.5)
    batch.set_collisions(0.5, 0.05, 60.0)
    x, v, f = _inputs(b, nat.FP32FORM)
    pen = []
    for s in range(30):
        got = _step(batch, nat.FP32FORM, x, v, f, b.iters)
        pen.append(_penetrations(b, got, x))
        x, v = got["x"], got["v"]
        assert np.all((got["status"] & 4) == 0)      # finite throughout
        assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    counts = [p[0] for p in pen]
    depths = [p[1] for p in pen]
    assert counts[0] > 500
    assert counts[1] < 0.85 * counts[0] and min(counts[1:4]) < 0.75 * counts[0], counts
    assert min(depths[1:4]) < 0.75 * depths[0], depths


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_packing_sampled(prec):
    """The 4096-RBC packing workload (642 vertices, 35 % volume fraction): detection of
    200 sampled vertices and the step of 2 sampled cells against the oracle."""
    nat = _native()
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = I.packing_batch(4096, 0, hematocrit=0.35, seed=1006)
    _, batch = _setup(b, p, radius=0.5)
    batch.set_collisions(0.5, 0.05, 60.0)
    x, v, f = _inputs(b, p)
    got = _step(batch, p, x, v, f, b.iters)
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    rng = np.random.default_rng(5)
    verts = sorted(int(i) for i in rng.choice(b.n_total, 200, replace=False))
    con = O.detect_contacts(ots, b.type_of_cell, b.offsets, x, 0.5, vertices=verts)
    _check_contacts(b, got, con, x, vertices=verts)
    cells = sorted(int(c) for c in rng.choice(b.ncells, 2, replace=False))
    ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, b.iters, cells=cells,
                       collisions=(0.5, 0.05, 60.0))
    assert _check_contacts(b, got, ref["contacts"], x,
                           vertices=[i for c in cells for i in range(b.offsets[c], b.offsets[c + 1])]) > 0
    _check_state(b, p, got, ref, cells, ots)


def test_collision_arguments_and_adjoint_rejected():
    nat = _native()
    b = _small_packing()
    _, batch = _setup(b, nat.FP64, collisions=False)
    for bad in ((0.0, 0.1, 1.0), (-1.0, 0.1, 1.0), (float("nan"), 0.1, 1.0), (float("inf"), 0.1, 1.0),
                (0.5, -0.1, 1.0), (0.5, 0.1, -1.0), (0.5, float("nan"), 1.0)):
        with pytest.raises(nat.NpfemError):
            batch.set_collisions(*bad)
    with pytest.raises(nat.NpfemError, match="never enabled"):
        batch.contacts(torch.zeros(b.n_total, dtype=torch.int32, device="cuda:0"))
    batch.set_collisions(RADIUS, DELTA, WEIGHT)
    dev = torch.device("cuda:0")
    X = torch.tensor(b.x, device=dev)
    g = [torch.zeros_like(X) for _ in range(5)]
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    with pytest.raises(nat.NpfemError, match="collisions"):
        batch.step_adjoint(X, X.clone(), X.clone(), g[0], g[1], g[2], g[3], g[4], gw, iters_default=3)


def test_contact_detection_timing():
    """With kernel timing on, the detection kernels' event pair gives a positive time,
    and timing leaves the step bit for bit unchanged."""
    nat = _native()
    b = _small_packing(seed=4)
    _, batch = _setup(b, nat.FP64)
    x, v, f = _inputs(b, nat.FP64)
    plain = _step(batch, nat.FP64, x, v, f, b.iters)
    with pytest.raises(nat.NpfemError, match="not timed"):
        batch.contact_time()
    batch.set_kernel_timing(True)
    timed = _step(batch, nat.FP64, x, v, f, b.iters)
    assert batch.contact_time() > 0.0
    for k in ("x", "v", "residual", "count", "vertex", "plane"):
        assert np.array_equal(plain[k], timed[k]), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_walls_parity(prec):
    """Small packing batch with the box walls of a cube that cuts into the cells: contacts
    plus wall penalties against the oracle, two steps."""
    nat = _native()
    p = nat.FP64 if prec == "fp64" else nat.FP32FORM
    b = _small_packing(seed=6)
    lo = b.x.min(axis=1) + 0.4
    hi = b.x.max(axis=1) - 0.4
    _, batch = _setup(b, p, collisions=False)
    batch.set_collisions(RADIUS, DELTA, WEIGHT, box=(lo, hi))
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    x, v, f = _inputs(b, p)
    for s in range(2):
        got = _step(batch, p, x, v, f, b.iters)
        ref = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, f, b.iters, collisions=(RADIUS, DELTA, WEIGHT),
                           box=(lo, hi))
        _check_contacts(b, got, ref["contacts"], x)
        _check_state(b, p, got, ref, range(b.ncells), ots)
        x, v = ref["x"], ref["v"]
        if p == nat.FP32FORM:
            x, v = (a.astype(np.float32).astype(np.float64) for a in (x, v))


def test_packing_in_a_box_stays_inside():
    """64 RBCs packed at 35 % volume fraction in a box whose walls sit 1 um outside the
    initial cells: after 30 steps no vertex is more than 0.2 um beyond a wall."""
    nat = _native()
    b = I.packing_batch(64, 0, hematocrit=0.35, seed=12)
    lo, hi = b.x.min(axis=1) - 1.0, b.x.max(axis=1) + 1.0
    _, batch = _setup(b, nat.FP32FORM, collisions=False)
    batch.set_collisions(0.5, 0.05, 60.0, box=(lo, hi))
    x, v, f = _inputs(b, nat.FP32FORM)
    worst = 0.0
    for s in range(30):
        got = _step(batch, nat.FP32FORM, x, v, f, b.iters)
        x, v = got["x"], got["v"]
        worst = max(worst, float(np.max(x - hi[:, None])), float(np.max(lo[:, None] - x)))
        assert np.all(np.isfinite(x))
    assert worst < 0.2, worst
