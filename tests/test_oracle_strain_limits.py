"""Pins of the oracle's strain-limit projection (singular values of each triangle's
deformation gradient clamped to [s_min, s_max]): the closed form against the SVD and,
at [1, 1], against the polar factor; exact energies of a uniaxial stretch and of an
isotropic scaling; the gradient and the complex-step derivative of a whole step against
central differences; rest invariance."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

MAT = (1.0, 0.05, 10.0, 10.0, 1.1)
DT = 0.1


def _random_F(rng, t):
    return rng.standard_normal((t, 3, 2)) * 0.4 + np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])


def _svd_project(F, lo, hi):
    out = np.empty_like(F)
    for t in range(F.shape[0]):
        U, s, Vt = np.linalg.svd(F[t], full_matrices=False)
        out[t] = U @ np.diag(np.clip(s, lo, hi)) @ Vt
    return out


@pytest.mark.parametrize("lo,hi", [(0.9, 1.1), (0.5, 1.0), (1.0, 1.5), (0.95, 1.05)])
def test_closed_form_matches_svd(lo, hi):
    F = _random_F(np.random.default_rng(61), 200)
    P, bad = O.clamped_project(F, lo, hi)
    assert not bad.any()
    assert np.allclose(P, _svd_project(F, lo, hi), rtol=0, atol=1e-12)


def test_closed_form_at_unit_limits_is_the_polar_factor():
    F = _random_F(np.random.default_rng(62), 200)
    P, _ = O.clamped_project(F, 1.0, 1.0)
    R, _ = O.polar_project(F)
    assert np.allclose(P, R, rtol=0, atol=1e-12)


def test_uniaxial_stretch_distance():
    rng = np.random.default_rng(63)
    lo, hi = 0.9, 1.1
    for lam in (0.7, 0.85, 0.95, 1.0, 1.05, 1.2, 1.6):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 2)))
        th = rng.uniform(0, 2 * np.pi)
        V = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        F = (Q @ np.diag([lam, 1.0]) @ V.T)[None]
        P, _ = O.clamped_project(F, lo, hi)
        d2 = float(np.sum((F - P) ** 2))
        want = (lam - hi) ** 2 if lam > hi else (lo - lam) ** 2 if lam < lo else 0.0
        assert d2 == pytest.approx(want, abs=1e-14), lam


@pytest.mark.parametrize("s", [0.8, 0.93, 1.0, 1.04, 1.25])
def test_isotropic_scaling_energy(s):
    """Scaling the rest mesh by s gives every triangle singular values (s, s), so the
    strain energy is w_strain A0 (s - clamp(s))^2."""
    lo, hi = 0.9, 1.1
    m = I.rbc_mesh(1)
    rs = O.rest_state(m.verts, m.tris, *MAT, DT, 0.0, 0.0, lo, hi)
    ctr = m.verts.mean(axis=0)
    parts, _ = O.internal_energy_and_gradient(rs, ctr + s * (m.verts - ctr))
    c = min(max(s, lo), hi)
    assert parts.strain == pytest.approx(MAT[0] * rs.A0 * (s - c) ** 2, rel=1e-10, abs=1e-14)


def test_limits_must_contain_the_rest_shape():
    m = I.icosahedron()
    for lo, hi in ((1.1, 1.2), (0.8, 0.9), (0.0, 1.1), (1.2, 1.1)):
        with pytest.raises(ValueError):
            O.rest_state(m.verts, m.tris, *MAT, DT, 0.0, 0.0, lo, hi)


def test_gradient_matches_central_differences():
    """Strain term alone (other weights 0), on a deformation with singular values
    below, inside and above the limits."""
    m = I.rbc_mesh(1)
    rs = O.rest_state(m.verts, m.tris, 1.0, 0.0, 0.0, 0.0, 1.1, DT, 0.0, 0.0, 0.95, 1.05)
    rng = np.random.default_rng(64)
    x = m.verts * np.array([1.08, 0.97, 1.0]) + 0.02 * rng.standard_normal(m.verts.shape)
    F = O.deformation_gradient(rs, x)
    sv = np.linalg.svd(F, compute_uv=False)
    assert np.any(sv > 1.05) and np.any(sv < 0.95) and np.any((sv > 0.95) & (sv < 1.05))
    _, g = O.internal_energy_and_gradient(rs, x)
    h = 1e-6
    for i, d in zip(rng.integers(0, m.n, 25), rng.integers(0, 3, 25)):
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        fd = (O.internal_energy_and_gradient(rs, xp)[0].strain
              - O.internal_energy_and_gradient(rs, xm)[0].strain) / (2 * h)
        assert g[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9), (i, d)


def test_rest_stays_at_rest_and_small_strains_are_free():
    """At rest nothing moves; a deformation whose singular values all lie inside the
    limits costs no strain energy, so (without bending, area and volume terms) the
    step keeps a free-flying cell's shape exactly like a rigid body."""
    m = I.rbc_mesh(1)
    ct = O.CellType(m.verts, m.tris, MAT + (0.0, 0.0, 0.9, 1.1), DT)
    x = m.verts + 3.0
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 5)
    assert np.max(np.abs(r.x - x)) < 1e-12
    soft = O.CellType(m.verts, m.tris, (1.0, 0.0, 0.0, 0.0, 1.1, 0.0, 0.0, 0.9, 1.1), DT)
    xs = m.verts * np.array([1.04, 0.98, 1.0])
    parts, g = O.internal_energy_and_gradient(soft.rest, xs)
    assert parts.strain == 0.0 and np.max(np.abs(g)) < 1e-14
    v = np.tile([0.3, -0.1, 0.2], (m.n, 1))
    r = O.step(soft.rest, soft.solver, xs, v, np.zeros_like(xs), 3)
    assert np.max(np.abs(r.x - (xs + DT * v))) < 1e-12


def test_complex_step_derivative_of_step_matches_central_differences():
    m = I.rbc_mesh(1)
    mat = MAT + (0.0, 0.0, 0.97, 1.03)
    ct = O.CellType(m.verts, m.tris, mat, DT)
    rng = np.random.default_rng(65)
    x = m.verts * np.array([1.06, 0.96, 1.0]) + 0.01 * rng.standard_normal(m.verts.shape)
    v = 0.05 * rng.standard_normal(x.shape)
    f = 0.1 * rng.standard_normal(x.shape)
    d = rng.standard_normal(x.shape)
    h, e = 1e-30, 1e-7
    cs = np.imag(O.step(ct.rest, ct.solver, x + 1j * h * d, v.astype(complex), f.astype(complex), 4).x) / h
    fd = (O.step(ct.rest, ct.solver, x + e * d, v, f, 4).x - O.step(ct.rest, ct.solver, x - e * d, v, f, 4).x) / (2 * e)
    assert np.max(np.abs(cs - fd)) <= 1e-5 * np.max(np.abs(cs))


def test_thin_triangles_project_accurately():
    """Nearly collapsed triangles (singular values (1.3, s2), s2 down to 1e-7, not flagged
    degenerate): the projection stays finite and agrees with the SVD to the closed
    form's own conditioning, about eps * s_min / s2 (the smaller eigenvalue det C / l1
    with det C = |F0 x F1|^2 has no cancellation; h - disc lost every digit of it here)."""
    rng = np.random.default_rng(71)
    lo, hi = 0.9, 1.1
    for s2 in (1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 2)))
        th = rng.uniform(0, 2 * np.pi)
        V = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        F = (Q @ np.diag([1.3, s2]) @ V.T)[None]
        P, bad = O.clamped_project(F, lo, hi)
        assert not bad.any() and np.all(np.isfinite(P))
        bound = 16 * np.finfo(float).eps * lo / s2 + 1e-14
        assert np.max(np.abs(P - _svd_project(F, lo, hi))) <= bound, s2
