"""Pins of the oracle's rest-state geometry against values fixed by geometry alone:
lumped masses worked out by hand, the hinge-stencil vector and magnitude in closed
form (dihedral angles and edge lengths), the bending energy written through those
angles, and the Evans-Fung cell's area and volume from quadrature of the smooth
surface.  None of the expected values is taken from the oracle's own arrays.

Readings pinned (Setting up new materials section: per-element energies and their
weights; the paper prints no formula):
* mass lumping: cell mass rho*V0 spread by the area share a third of the incident
  rest-triangle areas, m_i = rho V0 (sum_{t at i} A_t / 3) / A0;
* hinge stencil: for a hinge with edge (p0, p1) and opposite vertices p2 (triangle
  traversing p0 -> p1) and p3, K = sum_j c_j p_j with rest cotangent coefficients.
  For each of the two triangles, cot(angle at p1) (p0 - p_opp) + cot(angle at p0)
  (p1 - p_opp) = -|e| n, n the unit in-plane direction from the edge towards the
  opposite vertex, so K0 = -|e| (n_A + n_B) and |K0| = 2 |e| sin(theta/2), theta the
  angle between the two face normals (zero on a flat hinge, whatever its shape);
* bending weight w_e = w_bend * 3 / (A_A + A_B): with |K| = 2|e| sin(theta/2) the
  hinge energy is (w_bend/2) (3 |e|^2 / (A_A + A_B)) (2 sin(theta/2) - 2 sin(theta0/2))^2,
  the discrete-shells hinge energy of Grinspun et al. 2003 (|e|/h_e with
  h_e = (A_A + A_B)/(3|e|)) in its small-angle limit.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

MAT = (1.0, 0.05, 10.0, 10.0, 1.1)


def _rest(verts, tris, mat=MAT, dt=0.1):
    return O.rest_state(verts, tris, *mat, dt)


def _cube():
    v = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], float)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    return v, np.array(tris, np.int64)


def _corner_tetrahedron():
    """Vertices 0 = origin, 1..3 = the unit axis points; outward oriented faces."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    t = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int64)
    return v, t


def _random_tetrahedron(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((4, 3))
    t = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], np.int64)
    c = v.mean(axis=0)
    for i in range(4):          # outward orientation (a tetrahedron is convex)
        a, b, d = v[t[i]]
        if np.dot(np.cross(b - a, d - a), (a + b + d) / 3.0 - c) < 0:
            t[i, [1, 2]] = t[i, [2, 1]]
    return v, t


def _split_face_tetrahedron(seed):
    """A tetrahedron whose face (a, b, c) is split at a random interior point p into
    three coplanar, non-isosceles triangles: the hinges (a,p), (b,p), (c,p) are flat."""
    v, t = _random_tetrahedron(seed)
    rng = np.random.default_rng(seed + 1)
    lam = rng.dirichlet([2.0, 3.0, 4.0])
    a, b, c = t[3]
    p = lam[0] * v[a] + lam[1] * v[b] + lam[2] * v[c]
    v = np.vstack([v, p])
    ip = 4
    t = np.vstack([t[:3], [[a, b, ip], [b, c, ip], [c, a, ip]]])
    return v, t, {(min(a, ip), max(a, ip)), (min(b, ip), max(b, ip)), (min(c, ip), max(c, ip))}


# ------------------------------------------------------------ mass lumping
def test_lumped_masses_of_triangulated_cube_by_hand():
    """Unit cube, every face cut into two triangles of area 1/2: V0 = 1, A0 = 6.
    Counting incident triangles by hand (vertices 0 and 7 carry 6, the other six
    carry 4), m_i = rho * 1 * (k_i * 0.5 / 3) / 6 = rho k_i / 36."""
    v, t = _cube()
    rs = _rest(v, t)
    rho = MAT[4]
    expected = rho * np.array([6, 4, 4, 4, 4, 4, 4, 6]) / 36.0
    assert np.allclose(rs.mass, expected, rtol=1e-14, atol=0)


def test_lumped_masses_of_corner_tetrahedron_by_hand():
    """Origin + unit axis points: three right triangles of area 1/2 and one equilateral
    face of side sqrt(2) (area sqrt(3)/2); V0 = 1/6, A0 = 3/2 + sqrt(3)/2.  The origin
    touches the three right triangles (share 1/2), every other vertex two right
    triangles and the slanted face (share (1 + sqrt(3)/2)/3)."""
    v, t = _corner_tetrahedron()
    rs = _rest(v, t)
    rho = MAT[4]
    A0 = 1.5 + np.sqrt(3.0) / 2.0
    assert rs.A0 == pytest.approx(A0, rel=1e-15)
    assert rs.V0 == pytest.approx(1.0 / 6.0, rel=1e-14)
    share = np.array([0.5] + [(1.0 + np.sqrt(3.0) / 2.0) / 3.0] * 3)
    assert np.allclose(rs.mass, rho * (1.0 / 6.0) * share / A0, rtol=1e-14, atol=0)
    assert rs.mass[0] < rs.mass[1]          # a uniform split would give all four rho V0/4


# ------------------------------------------------------------ hinge stencil
def _hinge_geometry(X, hinges):
    """Per hinge (i, j, kA, kB): edge length, the two unit in-plane directions from the
    edge to the opposite vertices, the fold angle between the face normals, and the
    two triangle areas, all from positions by elementary geometry."""
    p0, p1, p2, p3 = (X[hinges[:, k]] for k in range(4))
    e = p1 - p0
    L = np.linalg.norm(e, axis=1)
    eh = e / L[:, None]

    def towards(p):
        d = p - p0
        d = d - np.sum(d * eh, axis=1)[:, None] * eh
        return d / np.linalg.norm(d, axis=1)[:, None]

    nA, nB = towards(p2), towards(p3)
    NA = np.cross(p1 - p0, p2 - p0)            # triangle (i, j, kA)
    NB = np.cross(p0 - p1, p3 - p1)            # triangle (j, i, kB)
    theta = np.arctan2(np.linalg.norm(np.cross(NA, NB), axis=1), np.sum(NA * NB, axis=1))
    areaA = 0.5 * np.linalg.norm(NA, axis=1)
    areaB = 0.5 * np.linalg.norm(NB, axis=1)
    return L, nA, nB, theta, areaA, areaB


MESHES = {
    "rbc_s2": lambda: (I.rbc_mesh(2).verts, I.rbc_mesh(2).tris),
    "random_tetrahedron": lambda: _random_tetrahedron(11),
    "corner_tetrahedron": _corner_tetrahedron,
    "split_face_tetrahedron": lambda: _split_face_tetrahedron(5)[:2],
    "platelet": lambda: (I.platelet_mesh().verts, I.platelet_mesh().tris),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_hinge_vector_closed_form(name):
    """K0 = -|e| (n_A + n_B) and |K0| = 2 |e| sin(theta/2) on every hinge."""
    X, t = MESHES[name]()
    rs = _rest(X, t)
    L, nA, nB, theta, _, _ = _hinge_geometry(np.asarray(X, float), rs.hinges)
    scale = np.max(L)
    assert np.allclose(rs.K0, -L[:, None] * (nA + nB), rtol=0, atol=1e-12 * scale)
    assert np.allclose(rs.kappa0, 2.0 * L * np.sin(theta / 2.0), rtol=0, atol=1e-12 * scale)


def test_asymmetric_flat_hinges_vanish():
    """The three hinges inside a split face are flat but have no symmetry (the
    triangles are not isosceles): the stencil must still annihilate them, and only
    them."""
    for seed in (5, 6, 7):
        X, t, flat = _split_face_tetrahedron(seed)
        rs = _rest(X, t)
        L, *_ = _hinge_geometry(X, rs.hinges)
        keys = [(int(h[0]), int(h[1])) for h in rs.hinges]
        is_flat = np.array([k in flat for k in keys])
        assert is_flat.sum() == 3
        assert np.all(rs.kappa0[is_flat] <= 1e-13 * np.max(L))
        assert np.all(rs.kappa0[~is_flat] > 1e-3 * np.max(L))
        # a stencil with the endpoint coefficients exchanged would leave
        # (c1 - c0)(p0 - p1) behind on these hinges: make sure that is not small
        c = rs.c_hinge[is_flat]
        assert np.all(np.abs(c[:, 1] - c[:, 0]) > 1e-3)


@pytest.mark.parametrize("s", [0.8, 1.1, 1.4])
@pytest.mark.parametrize("name", ["rbc_s2", "random_tetrahedron", "platelet"])
def test_bending_energy_in_dihedral_angles(name, s):
    """Isotropic scaling x = s X keeps every triangle's angles, so the hinge energy is
    (w_bend/2) (3 L^2 / (A_A + A_B)) (2 sin(theta/2))^2 (s - 1)^2 per hinge, with L,
    theta and the areas of the REST mesh measured geometrically."""
    X, t = MESHES[name]()
    X = np.asarray(X, float)
    rs = _rest(X, t)
    L, _, _, theta, aA, aB = _hinge_geometry(X, rs.hinges)
    c = X.mean(axis=0)
    parts, _ = O.internal_energy_and_gradient(rs, c + s * (X - c))
    w_bend = MAT[1]
    expected = np.sum(0.5 * w_bend * 3.0 * L ** 2 / (aA + aB) * (2.0 * np.sin(theta / 2.0)) ** 2) * (s - 1) ** 2
    assert parts.bend == pytest.approx(expected, rel=1e-11)


def test_bending_energy_of_a_folded_hinge():
    """Rotate the corner tetrahedron's vertex 3 about the x axis (the edge (0, 1)) by a
    small angle: both triangles at that edge stay congruent to their rest shapes, so
    the rest stencil gives |K| = 2 L sin(theta/2) at the new fold angle and the hinge's
    energy is (w_bend/2)(3 L^2/(A_A + A_B))(2 sin(theta/2) - 2 sin(theta0/2))^2."""
    X, t = _corner_tetrahedron()
    rs = _rest(X, t)
    keys = [(int(h[0]), int(h[1])) for h in rs.hinges]
    h01 = keys.index((0, 1))
    L, _, _, theta0, aA, aB = _hinge_geometry(X, rs.hinges)
    phi = 0.05
    Rx = np.array([[1, 0, 0], [0, np.cos(phi), -np.sin(phi)], [0, np.sin(phi), np.cos(phi)]])
    Y = X.copy()
    Y[3] = Rx @ X[3]                          # rotate vertex 3 about the x axis (edge 0-1)
    _, _, _, theta, _, _ = _hinge_geometry(Y, rs.hinges)
    # K of the hinge (0, 1) at Y from the rest stencil: both its triangles are congruent
    # to their rest shapes, so |K| = 2 L sin(theta/2) there
    cH = rs.c_hinge[h01]
    hh = rs.hinges[h01]
    K = sum(cH[k] * Y[hh[k]] for k in range(4))
    assert np.linalg.norm(K) == pytest.approx(2.0 * L[h01] * np.sin(theta[h01] / 2.0), rel=1e-13)
    assert abs(theta[h01] - theta0[h01]) == pytest.approx(phi, rel=1e-12)
    w_e = MAT[1] * 3.0 / (aA[h01] + aB[h01])
    e_expected = 0.5 * w_e * (2.0 * L[h01] * (np.sin(theta[h01] / 2.0) - np.sin(theta0[h01] / 2.0))) ** 2
    p = rs.kappa0[h01] * K / np.linalg.norm(K)
    assert 0.5 * rs.w_hinge[h01] * np.sum((K - p) ** 2) == pytest.approx(e_expected, rel=1e-12)


# ------------------------------------------------------------ Evans-Fung shape
def _evans_fung_exact(D=I.RBC_DIAMETER):
    """Area and volume of the smooth Evans-Fung surface by quadrature of its profile,
    parametrised by the polar angle phi of the sphere it is mapped from:
    r = (D/2) sin(phi), z = cos(phi) h(sin^2 phi), h(rho^2) = D (0.0518 + 2.0026 rho^2/4
    - 4.491 rho^4/16) (rho = 2r/D).  Area = int 2 pi r |(r', z')| dphi, volume =
    int pi r^2 (-z') dphi over [0, pi]."""
    R = D / 2.0

    def h(q):
        return D * (0.0518 + 2.0026 * q / 4.0 - 4.491 * q * q / 16.0)

    def dh(q):
        return D * (2.0026 / 4.0 - 2.0 * 4.491 * q / 16.0)

    def prof(p):
        s, c = np.sin(p), np.cos(p)
        return R * s, R * c, -s * h(s * s) + 2.0 * s * c * c * dh(s * s)

    area = integrate.quad(lambda p: 2 * np.pi * prof(p)[0] * np.hypot(prof(p)[1], prof(p)[2]), 0, np.pi,
                          epsabs=1e-12, epsrel=1e-13, limit=200)[0]
    vol = integrate.quad(lambda p: -np.pi * prof(p)[0] ** 2 * prof(p)[2], 0, np.pi,
                         epsabs=1e-12, epsrel=1e-13, limit=200)[0]
    return area, vol


def test_evans_fung_surface_area_and_volume():
    """The smooth shape has area 134.1 um^2 and volume 94.1 um^3; the s3 and s4 meshes
    are inscribed (smaller) and converge at second order in the edge length (the
    error falls by about 4 per subdivision)."""
    A, V = _evans_fung_exact()
    assert A == pytest.approx(134.1, abs=0.05)
    assert V == pytest.approx(94.1, abs=0.05)
    errs = []
    for s in (3, 4):
        m = I.rbc_mesh(s)
        rs = _rest(m.verts, m.tris)
        errs.append(((rs.A0 - A) / A, (rs.V0 - V) / V))
    (a3, v3), (a4, v4) = errs
    assert -0.01 < a3 < 0 and -0.012 < v3 < 0          # 642 vertices: within 1 % / 1.2 %
    assert -0.0025 < a4 < 0 and -0.003 < v4 < 0        # 2562 vertices: within 0.25 % / 0.3 %
    assert 3.5 < a3 / a4 < 4.5 and 3.5 < v3 / v4 < 4.5


def test_platelet_ellipsoid_volume():
    """The platelet is the s2 icosphere scaled to the semi-axes (1.8, 1.8, 0.5) um of an
    oblate ellipsoid of volume 4/3 pi 1.8^2 0.5 = 6.79 um^3; a linear map scales every
    volume by the same factor, so the mesh keeps the unit s2 icosphere's deficit."""
    m = I.platelet_mesh()
    rs = _rest(m.verts, m.tris)
    exact = 4.0 / 3.0 * np.pi * 1.8 * 1.8 * 0.5
    assert exact == pytest.approx(6.79, abs=0.005)
    unit = I.icosphere(2)
    rsu = _rest(unit.verts, unit.tris)
    deficit = rsu.V0 / (4.0 / 3.0 * np.pi)          # a linear map scales volumes uniformly
    assert rs.V0 == pytest.approx(exact * deficit, rel=1e-12)
    assert 0.95 < deficit < 1.0
