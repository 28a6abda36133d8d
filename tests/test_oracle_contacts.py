"""Pins of the oracle's collision reading: vertex normals, contact detection against an
independent KD-tree search, the contact penalty against central differences, the
impulse a contact delivers (closed form), force balance at a converged step, neutral
far planes, and overlapping cells separating."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

MAT = (1.0, 0.05, 10.0, 10.0, 1.1)
DT = 0.1


def _type(mesh, mat=MAT, dt=DT):
    return O.CellType(mesh.verts, mesh.tris, mat, dt)


def test_icosahedron_normals_are_radial():
    """By symmetry the area-weighted normal of a regular icosahedron's vertex is the
    radial direction; rotating the mesh rotates the normals."""
    m = I.icosahedron()
    n = O.vertex_normals(m.verts, m.tris)
    assert np.allclose(n, m.verts / np.linalg.norm(m.verts, axis=1, keepdims=True), rtol=0, atol=1e-14)
    R = I.random_rotation(np.random.default_rng(3))
    assert np.allclose(O.vertex_normals(m.verts @ R.T, m.tris), n @ R.T, rtol=0, atol=1e-14)


def test_rbc_normals_are_volume_gradient_directions():
    """For a closed mesh dV/dx_i = (1/6) sum over incident triangles of (x1-x0)x(x2-x0)
    (the fan's other terms cancel), so the unit normal is the direction of the
    enclosed volume's gradient: checked by central differences on the biconcave RBC
    (V is linear in each coordinate of one vertex, so the differences are exact up to
    rounding for any step)."""
    m = I.rbc_mesh(2)
    n = O.vertex_normals(m.verts, m.tris)
    h = 1e-3
    for i in range(0, m.n, 5):
        gv = np.zeros(3)
        for d in range(3):
            xp, xm = m.verts.copy(), m.verts.copy()
            xp[i, d] += h
            xm[i, d] -= h
            gv[d] = (O._volume(xp, m.tris) - O._volume(xm, m.tris)) / (2 * h)
        assert np.allclose(gv / np.linalg.norm(gv), n[i], rtol=0, atol=1e-10)


def _overlapping_spheres(seed=5, ncells=6, box=3.0, subdiv=1):
    types = [I.CellTypeSpec(I.icosphere(subdiv), I.RBC_MATERIAL)]
    rng = np.random.default_rng(seed)
    xs = [I.icosphere(subdiv).verts @ I.random_rotation(rng).T + rng.uniform(0, box, 3) for _ in range(ncells)]
    z = [np.zeros_like(x) for x in xs]
    return I._assemble(types, [0] * ncells, xs, z, z, [4] * ncells, DT, seed)


def test_detection_matches_kdtree_search():
    """Brute-force detection equals an independent search: a KD-tree ball query, the
    nearest vertex per other cell, the two nearest cells kept."""
    from scipy.spatial import cKDTree
    b = _overlapping_spheres()
    ots = [_type(t.mesh) for t in b.types]
    radius = 0.6
    con = O.detect_contacts(ots, b.type_of_cell, b.offsets, b.x, radius)
    cell_of = np.repeat(np.arange(b.ncells), np.diff(b.offsets))
    tree = cKDTree(b.x.T)
    total = 0
    for i in range(b.n_total):
        best = {}
        for j in tree.query_ball_point(b.x[:, i], radius * (1 + 1e-9)):
            cb = int(cell_of[j])
            if cb == cell_of[i]:
                continue
            d = float(np.linalg.norm(b.x[:, i] - b.x[:, j]))
            if d < radius and (cb not in best or (d, j) < best[cb]):
                best[cb] = (d, j)
        kept = sorted(((d, cb, j) for cb, (d, j) in best.items()))[:2]
        assert con["count"][i] == len(kept)
        for k, (d, cb, j) in enumerate(kept):
            assert (con["cell"][i, k], con["vertex"][i, k]) == (cb, j)
            nb = O.vertex_normals(b.x[:, b.cell_slice(cb)].T, b.types[0].mesh.tris)[j - b.offsets[cb]]
            assert np.allclose(con["normal"][i, k], nb, rtol=0, atol=1e-15)
            assert con["offset"][i, k] == pytest.approx(float(nb @ b.x[:, j]), rel=0, abs=1e-14)
        total += len(kept)
    assert total > 50          # the configuration really overlaps


def test_equal_distances_go_to_the_smaller_cell():
    """A vertex of cell 0 on the plane x = 0, with cell 2 the mirror image of cell 1 in that
    plane: its nearest vertices in cells 1 and 2 are at exactly equal distances, and the
    tie goes to the smaller cell index (slot 0 = cell 1, slot 1 = cell 2)."""
    m = I.icosphere(1)
    x0 = m.verts.copy()
    x1 = m.verts + np.array([1.5, 0.0, 0.0])
    x2 = x1 * np.array([-1.0, 1.0, 1.0])
    z = [np.zeros_like(x0)] * 3
    b = I._assemble([I.CellTypeSpec(m, I.RBC_MATERIAL)], [0, 0, 0], [x0, x1, x2], z, z, [1] * 3, DT, 0)
    ots = [_type(t.mesh) for t in b.types]
    con = O.detect_contacts(ots, b.type_of_cell, b.offsets, b.x, 1.0)
    on_plane = np.flatnonzero(x0[:, 0] == 0.0)
    assert len(on_plane) > 0
    ties = 0
    for i in on_plane:
        if con["count"][i] == 2:
            j1, j2 = con["vertex"][i]
            assert list(con["cell"][i]) == [1, 2]
            assert j2 - b.offsets[2] == j1 - b.offsets[1]      # mirror images of one vertex
            ties += 1
    assert ties > 0


def test_detection_is_translation_invariant():
    b = _overlapping_spheres(seed=8)
    ots = [_type(t.mesh) for t in b.types]
    c0 = O.detect_contacts(ots, b.type_of_cell, b.offsets, b.x, 0.6)
    t = np.array([[64.0], [-32.0], [16.0]])    # exact in binary: distances unchanged
    c1 = O.detect_contacts(ots, b.type_of_cell, b.offsets, b.x + t, 0.6)
    for k in ("count", "vertex", "cell"):
        assert np.array_equal(c0[k], c1[k])
    assert np.allclose(c0["normal"], c1["normal"], rtol=0, atol=1e-12)
    used = c0["vertex"] >= 0
    shift = np.einsum("nkd,d->nk", c0["normal"], t[:, 0])
    assert np.allclose(c1["offset"][used], (c0["offset"] + shift)[used], rtol=0, atol=1e-12)


def test_contact_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((20, 3))
    idx = np.array([0, 3, 3, 7, 12, 19])
    nrm = rng.standard_normal((6, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    crel = np.sum(nrm * x[idx], axis=1) + rng.uniform(-0.4, 0.4, 6)   # gaps in [-0.4, 0.4]
    delta, w = 0.1, 7.0
    E, g = O.contact_energy_and_gradient(x, idx, nrm, crel, delta, w)
    assert E > 0
    h = 1e-6
    for v in range(20):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, d] += h
            xm[v, d] -= h
            fd = (O.contact_energy_and_gradient(xp, idx, nrm, crel, delta, w)[0]
                  - O.contact_energy_and_gradient(xm, idx, nrm, crel, delta, w)[0]) / (2 * h)
            assert g[v, d] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_far_planes_leave_the_step_unchanged():
    """Planes that no iterate comes within delta of add exactly zero energy and
    gradient: the step is bit-identical to the step without contacts."""
    b = I.single_rbc(subdiv=2)
    ct = _type(b.types[0].mesh)
    x, v, f = b.cell_state(0)
    f = 20 * f
    r0 = O.step(ct.rest, ct.solver, x, v, f, 5)
    idx = np.arange(0, x.shape[0], 7)
    nrm = np.tile([0.0, 0.0, 1.0], (len(idx), 1))
    c_abs = x[idx, 2] - 50.0                    # planes 50 um below each vertex
    r1 = O.step(ct.rest, ct.solver, x, v, f, 5, contact=(idx, nrm, c_abs, 0.2, 30.0))
    assert np.array_equal(r0.x, r1.x) and np.array_equal(r0.v, r1.v)


def test_one_contact_delivers_its_impulse():
    """A rest cell with one penetrating contact: the first quasi-Newton iterate is
    the PD step d = -A^-1 g, and since A 1 = m/dt^2 (the elastic blocks annihilate
    translations), the mass-weighted displacement equals dt^2 w (delta - gap) n."""
    m = I.rbc_mesh(2)
    ct = _type(m)
    x = m.verts.copy()
    i = 17
    n = np.array([0.6, 0.0, 0.8])
    gap = -0.3
    c_abs = float(n @ x[i]) - gap
    delta, w = 0.1, 25.0
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 1,
               contact=(np.array([i]), n[None, :], np.array([c_abs]), delta, w))
    impulse = np.sum(ct.rest.mass[:, None] * (r.x - x), axis=0)
    assert np.allclose(impulse, DT * DT * w * (delta - gap) * n, rtol=1e-12, atol=1e-15)


def test_converged_step_balances_contact_forces():
    """At the minimiser the elastic forces sum to zero, so the inertial term balances
    the contact forces: sum_i m_i (x_i - y_i) / dt^2 = w sum_k max(0, delta - gap_k) n_k."""
    m = I.icosphere(2)
    ct = _type(m, dt=0.5)
    rng = np.random.default_rng(4)
    x = m.verts * 2.0
    idx = np.array([3, 40, 41, 100])
    nrm = rng.standard_normal((4, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    c_abs = np.sum(nrm * x[idx], axis=1) + 0.05
    delta, w = 0.1, 3.0
    con = (idx, nrm, c_abs, delta, w)
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 300, contact=con)
    assert r.residual < 1e-10
    lhs = np.sum(ct.rest.mass[:, None] * (r.x - x), axis=0) / 0.25
    gap = np.sum(nrm * r.x[idx], axis=1) - c_abs
    rhs = w * np.sum(np.maximum(0.0, delta - gap)[:, None] * nrm, axis=0)
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-12)


def test_overlapping_cells_separate():
    """Two unit spheres overlapping by 0.4 um at rest: without contacts nothing moves;
    with contacts each step reduces the number of vertices inside the other sphere."""
    m = I.icosphere(2)
    types = [I.CellTypeSpec(m, I.RBC_MATERIAL)]
    xa, xb = m.verts.copy(), m.verts + np.array([1.6, 0.0, 0.0])
    z = np.zeros_like(xa)
    b = I._assemble(types, [0, 0], [xa, xb], [z, z], [z, z], [5, 5], 0.1, 0)
    ots = [_type(m)]

    def inside():
        ca, cb = b.x[:, :m.n].mean(axis=1), b.x[:, m.n:].mean(axis=1)
        return (int(np.sum(np.linalg.norm(b.x[:, :m.n] - cb[:, None], axis=0) < 0.999))
                + int(np.sum(np.linalg.norm(b.x[:, m.n:] - ca[:, None], axis=0) < 0.999)))

    r = O.batch_step(ots, b.type_of_cell, b.offsets, b.x, b.v, b.f, b.iters)
    assert np.allclose(r["x"], b.x, rtol=0, atol=1e-14)
    counts = [inside()]
    x, v = b.x.copy(), b.v.copy()
    for _ in range(6):
        r = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, b.f, b.iters, collisions=(0.5, 0.1, 50.0))
        x, v = r["x"], r["v"]
        b.x = x
        counts.append(inside())
    assert counts[0] > 0
    assert all(c1 <= c0 for c0, c1 in zip(counts, counts[1:])) and counts[-1] < counts[0]


def test_wall_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    x = rng.uniform(-1.0, 1.0, (30, 3))
    lo, hi = np.array([-0.9, -0.8, -1.0]), np.array([0.85, 0.9, 0.7])
    E, g = O.wall_energy_and_gradient(x, lo, hi, 0.2, 9.0)
    assert E > 0
    h = 1e-6
    for v in range(30):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, d] += h
            xm[v, d] -= h
            fd = (O.wall_energy_and_gradient(xp, lo, hi, 0.2, 9.0)[0]
                  - O.wall_energy_and_gradient(xm, lo, hi, 0.2, 9.0)[0]) / (2 * h)
            assert g[v, d] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_one_wall_contact_delivers_its_impulse():
    """A rest cell with one vertex a distance p beyond the lower x wall and every other
    vertex farther than delta inside: the first PD iterate's mass-weighted displacement is
    dt^2 w (delta + p) along +x (as for one cell contact)."""
    m = I.rbc_mesh(2)
    ct = _type(m)
    x = m.verts.copy()
    order = np.argsort(x[:, 0])
    p, delta, w = 0.05, 0.02, 25.0
    lo = np.array([x[order[0], 0] + p, -100.0, -100.0])
    hi = np.array([100.0, 100.0, 100.0])
    assert x[order[1], 0] > lo[0] + delta
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 1, walls=(lo, hi, delta, w))
    impulse = np.sum(ct.rest.mass[:, None] * (r.x - x), axis=0)
    assert np.allclose(impulse, DT * DT * w * (delta + p) * np.array([1.0, 0.0, 0.0]), rtol=1e-12, atol=1e-15)


def test_cell_thrown_at_a_wall_turns_back():
    """A cell moving at 2 um/us towards the upper x wall: within a few steps its velocity
    turns negative and no vertex gets more than 0.3 um beyond the wall."""
    m = I.icosphere(2)
    ct = _type(m)
    x = m.verts.copy()
    v = np.tile([[2.0, 0.0, 0.0]], (m.n, 1))
    lo, hi = np.array([-5.0, -5.0, -5.0]), np.array([1.5, 5.0, 5.0])
    worst = 0.0
    for _ in range(20):
        r = O.step(ct.rest, ct.solver, x, v, np.zeros_like(x), 8, walls=(lo, hi, 0.05, 200.0))
        x, v = r.x, r.v
        worst = max(worst, float(np.max(x[:, 0] - hi[0])))
    assert np.mean(v[:, 0]) < 0
    assert worst < 0.3
