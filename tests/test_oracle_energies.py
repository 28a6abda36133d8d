"""Pins of the oracle's energies, projections, rest state and global matrix against
closed forms, invariants and finite differences (nothing here reuses the formula
under test to produce its expected value)."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

MAT = (1.0, 0.05, 10.0, 10.0, 1.1)


def _rest(mesh, mat=MAT, dt=0.1):
    return O.rest_state(mesh.verts, mesh.tris, *mat, dt)


def _rand_rot(seed):
    return I.random_rotation(np.random.default_rng(seed))


@pytest.fixture(scope="module")
def rbc2():
    return I.rbc_mesh(2)


# ------------------------------------------------------------ closed forms
def test_regular_tetrahedron_area_volume():
    m = I.tetrahedron()           # circumradius 1
    rs = _rest(m)
    a = 4.0 / np.sqrt(6.0)        # edge length of the regular tetrahedron
    assert rs.A0 == pytest.approx(np.sqrt(3.0) * a * a, rel=1e-14)
    assert rs.V0 == pytest.approx(a ** 3 / (6.0 * np.sqrt(2.0)), rel=1e-14)
    assert np.sum(rs.mass) == pytest.approx(MAT[4] * rs.V0, rel=1e-14)
    # regular: every vertex carries a quarter of the mass
    assert np.allclose(rs.mass, MAT[4] * rs.V0 / 4.0, rtol=1e-14)


def test_cell_collapsed_to_a_point():
    """Every vertex at one point: each triangle is degenerate (F = 0, no strain energy, and
    counted), each hinge has K = 0 exactly and falls back to p = K0, so the bending energy
    is sum_e (w_e/2)|K0_e|^2; A = V = 0 leaves (w_A/2) A0 and (w_V/2) V0."""
    m = I.rbc_mesh(2)
    rs = _rest(m)
    x = np.tile(np.array([[1.5, -2.0, 0.7]]), (m.n, 1))
    parts, _ = O.internal_energy_and_gradient(rs, x)
    assert parts.strain == 0.0
    assert parts.degenerate == m.ntris
    assert parts.bend == pytest.approx(0.5 * np.sum(rs.w_hinge * np.sum(rs.K0 * rs.K0, axis=1)), rel=1e-14)
    assert parts.bend > 0.0
    assert parts.area == pytest.approx(0.5 * MAT[2] * rs.A0, rel=1e-14)
    assert parts.volume == pytest.approx(0.5 * MAT[3] * rs.V0, rel=1e-14)


def test_icosphere_counts_and_sphere_limits():
    for s in range(4):
        m = I.icosphere(s)
        assert m.n == 10 * 4 ** s + 2 and m.ntris == 20 * 4 ** s
        assert O.hinges_of(m.tris, m.n).shape[0] == 30 * 4 ** s
    rs = _rest(I.icosphere(4))
    assert rs.A0 == pytest.approx(4 * np.pi, rel=2e-3)
    assert rs.V0 == pytest.approx(4 * np.pi / 3, rel=4e-3)


@pytest.mark.parametrize("s", [0.9, 1.05, 1.3])
def test_isotropic_scaling_energies(rbc2, s):
    """x = s*(X - c): every F has singular values (s, s), so E_strain = w A0 (s-1)^2;
    |K| = s|K0| gives E_bend = sum w_e/2 (s-1)^2 |K0|^2; A = s^2 A0, V = s^3 V0."""
    rs = _rest(rbc2)
    X = rbc2.verts
    c = X.mean(axis=0)
    x = c + s * (X - c)
    parts, _ = O.internal_energy_and_gradient(rs, x)
    assert parts.strain == pytest.approx(MAT[0] * rs.A0 * (s - 1) ** 2, rel=1e-12)
    assert parts.bend == pytest.approx(np.sum(0.5 * rs.w_hinge * rs.kappa0 ** 2) * (s - 1) ** 2,
                                       rel=1e-12)
    assert parts.A == pytest.approx(s * s * rs.A0, rel=1e-13)
    assert parts.V == pytest.approx(s ** 3 * rs.V0, rel=1e-13)
    assert parts.area == pytest.approx(0.5 * MAT[2] * (s * s - 1) ** 2 * rs.A0, rel=1e-12)
    assert parts.volume == pytest.approx(0.5 * MAT[3] * (s ** 3 - 1) ** 2 * rs.V0, rel=1e-12)


def test_uniaxial_stretch_polar():
    """F = Q diag-like(lambda, 1) P: projection is Q[[1,0],[0,1],[0,0]]P and
    |F - R|^2 / 2 = (lambda - 1)^2 / 2."""
    rng = np.random.default_rng(3)
    for lam in (0.5, 1.0, 1.7, 3.0):
        Q = _rand_rot(int(rng.integers(1 << 30)))
        th = rng.uniform(0, 2 * np.pi)
        P = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        base = np.array([[lam, 0.0], [0.0, 1.0], [0.0, 0.0]])
        F = (Q @ base @ P)[None]
        R, bad = O.polar_project(F)
        assert not bad.any()
        Rexp = Q @ np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]]) @ P
        assert np.allclose(R[0], Rexp, atol=1e-14)
        assert 0.5 * np.sum((F[0] - R[0]) ** 2) == pytest.approx(0.5 * (lam - 1) ** 2, abs=1e-14)


def test_polar_matches_svd():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((50, 3, 2))
    R, _ = O.polar_project(F)
    for i in range(50):
        U, _, Vt = np.linalg.svd(F[i], full_matrices=False)
        assert np.allclose(R[i], U @ Vt, atol=1e-12)


def test_degenerate_triangle_flagged():
    F = np.zeros((1, 3, 2))
    F[0, 0, 0] = 1.0        # rank one
    R, bad = O.polar_project(F)
    assert bad[0] and np.array_equal(R, F)


def test_hinge_stencil_sums_to_zero():
    """sum_j c_j = 0, so K is invariant under translation."""
    rs = _rest(I.rbc_mesh(2))
    assert np.allclose(rs.c_hinge.sum(axis=1), 0.0, atol=1e-12)


def _cube():
    v = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], float)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    return I.Mesh(v, np.array(tris, np.int32), "cube")


def test_flat_hinges_of_closed_mesh_vanish():
    """On a triangulated cube the six face diagonals are flat hinges: the cotangent
    stencil annihilates them (K0 = 0), while the twelve cube edges are bent."""
    m = _cube()
    rs = _rest(m)
    assert rs.hinges.shape[0] == 18
    assert rs.V0 == pytest.approx(1.0, rel=1e-14) and rs.A0 == pytest.approx(6.0, rel=1e-14)
    flat = rs.kappa0 < 1e-12
    assert int(np.sum(flat)) == 6
    assert np.min(rs.kappa0[~flat]) > 0.5


# ------------------------------------------------------------ invariants
def _deformed(m, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    return m.verts + amp * rng.standard_normal(m.verts.shape)


def test_rest_energy_and_gradient_zero(rbc2):
    rs = _rest(rbc2)
    parts, g = O.internal_energy_and_gradient(rs, rbc2.verts)
    assert parts.strain < 1e-26 and parts.bend < 1e-26
    assert parts.area < 1e-26 and parts.volume < 1e-24
    assert np.max(np.abs(g)) < 1e-12


def test_momentum_conservation(rbc2):
    """Internal forces sum to zero and exert no net torque (linear/angular momentum)."""
    rs = _rest(rbc2)
    x = _deformed(rbc2, 1)
    _, g = O.internal_energy_and_gradient(rs, x)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(g.sum(axis=0))) < 1e-12 * scale * rbc2.n
    torque = np.cross(x, g).sum(axis=0)
    assert np.max(np.abs(torque)) < 1e-11 * scale * rbc2.n


def test_rigid_motion_invariance(rbc2):
    rs = _rest(rbc2)
    x = _deformed(rbc2, 2)
    Q = _rand_rot(9)
    t = np.array([150.0, -20.0, 75.0])
    p1, g1 = O.internal_energy_and_gradient(rs, x)
    p2, g2 = O.internal_energy_and_gradient(rs, x @ Q.T + t)
    for a, b in ((p1.strain, p2.strain), (p1.bend, p2.bend), (p1.area, p2.area),
                 (p1.volume, p2.volume)):
        assert b == pytest.approx(a, rel=1e-10, abs=1e-18)
    assert np.allclose(g2, g1 @ Q.T, rtol=0, atol=1e-10 * np.max(np.abs(g1)))


@pytest.mark.parametrize("mesh_fn", [I.tetrahedron, I.icosahedron, lambda: I.rbc_mesh(1),
                                     lambda: I.platelet_mesh(1)])
def test_gradient_matches_central_differences(mesh_fn):
    m = mesh_fn()
    rs = _rest(m)
    rng = np.random.default_rng(11)
    x = m.verts + 0.08 * rng.standard_normal(m.verts.shape) * np.ptp(m.verts)
    y = m.verts + 0.02 * rng.standard_normal(m.verts.shape)
    _, g = O.objective(rs, x, y)
    for trial in range(3):
        dvec = rng.standard_normal(x.shape)
        h = 1e-6
        fp = O.objective(rs, x + h * dvec, y)[0].total
        fm = O.objective(rs, x - h * dvec, y)[0].total
        fd = (fp - fm) / (2 * h)
        an = np.sum(g * dvec)
        assert fd == pytest.approx(an, rel=1e-7, abs=1e-9 * np.abs(g).sum())


# ------------------------------------------------------------ global matrix
def test_pd_matrix_structure(rbc2):
    rs = _rest(rbc2)
    A = O.pd_matrix(rs)
    assert np.allclose(A, A.T, atol=0)
    assert np.min(np.linalg.eigvalsh(A)) > 0
    # rigid translation is in the kernel of every elastic block: A 1 = m/dt^2
    assert np.allclose(A @ np.ones(rs.n), rs.mass / rs.dt ** 2, rtol=1e-12, atol=1e-9)


def test_pd_matrix_is_hessian_of_pd_quadratic(rbc2):
    """A u = gradient of the PD quadratic u^T M u/(2dt^2) + sum_t w_t/2 |F(u)|^2 +
    sum_e w_e/2 |K(u)|^2, with F and K linear in u (differenced numerically)."""
    rs = _rest(rbc2)
    A = O.pd_matrix(rs)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((rs.n, 3))

    def quad(z):
        F = O.deformation_gradient(rs, z)
        K = O.hinge_K(rs, z)
        return (np.sum(rs.mass[:, None] * z * z) / (2 * rs.dt ** 2)
                + 0.5 * np.sum(rs.w_tri * np.einsum("tij,tij->t", F, F))
                + 0.5 * np.sum(rs.w_hinge * np.einsum("ij,ij->i", K, K)))

    dvec = rng.standard_normal((rs.n, 3))
    h = 1e-4
    fd = (quad(u + h * dvec) - quad(u - h * dvec)) / (2 * h)     # exact for a quadratic
    an = np.sum((A @ u) * dvec)
    assert fd == pytest.approx(an, rel=1e-9)


def test_global_solver_matches_dense_solve(rbc2):
    rs = _rest(rbc2)
    A = O.pd_matrix(rs)
    gs = O.GlobalSolver(A)
    q = np.random.default_rng(13).standard_normal((rs.n, 3))
    assert np.allclose(gs.solve(q), np.linalg.solve(A, q), rtol=1e-12, atol=1e-14)
