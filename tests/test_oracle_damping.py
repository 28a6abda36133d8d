"""Pins of the oracle's damping reading (Rayleigh damping C = c_alpha M + c_beta L, L
the elastic part of the projective-dynamics matrix, in implicit Euler): the exact
decay of a rigid motion, translation invariance of the c_beta part, the one-iteration
damped projective-dynamics step assembled independently, the gradient against central
differences, and dissipation of mechanical energy."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

DT = 0.1


def _type(mesh, mat):
    return O.CellType(mesh.verts, mesh.tris, mat, DT)


def test_mass_damping_slows_a_rigid_motion_exactly():
    """A rest-shaped cell moving rigidly with velocity v, no force: the step solves
    (M/dt^2 + c_alpha M/dt)(x - x_n) = M v / dt, so v_{n+1} = v / (1 + c_alpha dt),
    already after one quasi-Newton iteration (the PD step is exact on this quadratic)."""
    m = I.rbc_mesh(2)
    alpha = 0.7
    ct = _type(m, (1.0, 0.05, 10.0, 10.0, 1.1, alpha, 0.0))
    v = np.tile(np.array([[0.3, -0.1, 0.2]]), (m.n, 1))
    for iters in (1, 5):
        r = O.step(ct.rest, ct.solver, m.verts, v, np.zeros_like(v), iters)
        assert np.allclose(r.v, v / (1.0 + alpha * DT), rtol=0, atol=1e-12)
        assert np.allclose(r.x, m.verts + DT * v / (1.0 + alpha * DT), rtol=0, atol=1e-13)


def test_stiffness_damping_leaves_translations_alone():
    """L annihilates translations, so c_beta damping does not slow a rigid translation."""
    m = I.rbc_mesh(2)
    ct = _type(m, (1.0, 0.05, 10.0, 10.0, 1.1, 0.0, 2.5))
    v = np.tile(np.array([[0.3, -0.1, 0.2]]), (m.n, 1))
    r = O.step(ct.rest, ct.solver, m.verts, v, np.zeros_like(v), 3)
    assert np.allclose(r.v, v, rtol=0, atol=1e-11)


def test_one_iteration_equals_damped_projective_dynamics_step():
    """No area/volume energy, one iteration: x1 = A'^-1 (M y/dt^2 + C x_n/dt + sum_t w_t
    G_t^T p_t + sum_e w_e c_e p_e) with A' = M/dt^2 + L + C/dt, both assembled here
    from the element blocks."""
    m = I.rbc_mesh(2)
    alpha, beta = 0.4, 0.8
    ct = _type(m, (1.0, 0.05, 0.0, 0.0, 1.1, alpha, beta))
    rs = ct.rest
    rng = np.random.default_rng(23)
    x = m.verts
    v = 0.5 * rng.standard_normal(x.shape)
    f = 0.05 * rng.standard_normal(x.shape)
    r = O.step(rs, ct.solver, x, v, f, 1)
    assert r.alphas == [1.0]
    y = x + DT * v + DT * DT * f / rs.mass[:, None]
    Fy = O.deformation_gradient(rs, y)
    P, _ = O.polar_project(Fy)
    n = rs.n
    L = np.zeros((n, n))
    rhs = rs.mass[:, None] * y / DT ** 2
    S = np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
    for t in range(rs.tris.shape[0]):
        G = rs.Dm_inv[t].T @ S
        L[np.ix_(rs.tris[t], rs.tris[t])] += rs.w_tri[t] * (G.T @ G)
        np.add.at(rhs, rs.tris[t], rs.w_tri[t] * G.T @ P[t].T)
    K = O.hinge_K(rs, y)
    p = O.bending_project(rs, K)
    for e in range(rs.hinges.shape[0]):
        c = rs.c_hinge[e]
        L[np.ix_(rs.hinges[e], rs.hinges[e])] += rs.w_hinge[e] * np.outer(c, c)
        np.add.at(rhs, rs.hinges[e], rs.w_hinge[e] * np.outer(c, p[e]))
    M = np.diag(rs.mass)
    C = alpha * M + beta * L
    rhs = rhs + C @ x / DT
    x1 = np.linalg.solve(M / DT ** 2 + L + C / DT, rhs)
    assert np.allclose(r.x, x1, rtol=0, atol=1e-12 * np.max(np.abs(x1)))


def test_damped_gradient_matches_central_differences():
    m = I.icosphere(1)
    ct = _type(m, (1.0, 0.05, 10.0, 10.0, 1.1, 0.6, 0.9))
    rs = ct.rest
    rng = np.random.default_rng(29)
    xn = m.verts + 0.05 * rng.standard_normal(m.verts.shape)
    y = xn + 0.1 * rng.standard_normal(m.verts.shape)
    x = y + 0.05 * rng.standard_normal(m.verts.shape)
    damp = (xn, O.damping_matrix(rs))
    parts, g = O.objective(rs, x, y, None, None, damp)
    assert parts.damping > 0
    h = 1e-6
    for i in range(m.n):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (O.objective(rs, xp, y, None, None, damp)[0].total
                  - O.objective(rs, xm, y, None, None, damp)[0].total) / (2 * h)
            assert g[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def _mechanical_energy(rs, x, v):
    parts, _ = O.internal_energy_and_gradient(rs, x - x.mean(axis=0))
    return 0.5 * float(np.sum(rs.mass[:, None] * v * v)) + parts.strain + parts.bend + parts.area + parts.volume


def test_damping_dissipates_mechanical_energy():
    """A cell stretched along x and released at rest: with Rayleigh damping its kinetic
    plus elastic energy never grows from step to step and ends below the undamped run's."""
    m = I.rbc_mesh(2)
    x0 = m.verts * np.array([1.15, 0.95, 0.95])
    ends = []
    for mat in ((1.0, 0.05, 10.0, 10.0, 1.1, 0.0, 0.0), (1.0, 0.05, 10.0, 10.0, 1.1, 0.5, 1.0)):
        ct = _type(m, mat)
        x, v = x0.copy(), np.zeros_like(x0)
        energies = [_mechanical_energy(ct.rest, x, v)]
        for _ in range(12):
            r = O.step(ct.rest, ct.solver, x, v, np.zeros_like(x), 8)
            x, v = r.x, r.v
            energies.append(_mechanical_energy(ct.rest, x, v))
        ends.append(energies[-1])
        if mat[5] > 0:
            e = np.array(energies)
            assert np.all(e[1:] <= e[:-1] * (1 + 1e-9)), e
    assert ends[1] < ends[0]


def test_damped_complex_step_derivative_matches_central_differences():
    """The oracle's forward-mode derivative of the damped step (complex step through the
    whole fixed-iteration step) agrees with central differences of the real step, for
    perturbations of x_n (which the dissipation term sees directly), v_n, f and the weight
    scales (which also scale the c_beta part of C and of the solver's matrix)."""
    mat = (1.0, 0.05, 10.0, 10.0, 1.1, 0.5, 1.0)
    m = I.rbc_mesh(1)
    rng = np.random.default_rng(31)
    x = m.verts * np.array([1.1, 0.95, 1.0]) + 0.02 * rng.standard_normal(m.verts.shape) + 3.0
    v = 0.1 * rng.standard_normal(x.shape)
    f = 0.2 * rng.standard_normal(x.shape)
    ct = _type(m, mat)
    iters, h, e = 5, 1e-30, 1e-6

    def step(xx, vv, ff, ws=None, c=ct):
        return O.step(c.rest, c.solver, xx, vv, ff, iters, ws)

    for name in ("x", "v", "f"):
        d = rng.standard_normal(x.shape)
        arg = {"x": x, "v": v, "f": f}
        cplx = {k: a.astype(complex) for k, a in arg.items()}
        cplx[name] = arg[name] + 1j * h * d
        r = step(cplx["x"], cplx["v"], cplx["f"])
        cs = np.imag(r.x) / h
        hi = dict(arg)
        lo = dict(arg)
        hi[name] = arg[name] + e * d
        lo[name] = arg[name] - e * d
        fd = (step(hi["x"], hi["v"], hi["f"]).x - step(lo["x"], lo["v"], lo["f"]).x) / (2 * e)
        assert np.max(np.abs(cs - fd)) <= 1e-6 * np.max(np.abs(cs)), name
    for q in range(4):
        ws = np.ones(4, complex)
        ws[q] += 1j * h
        ctc = O.CellType(m.verts, m.tris, mat, DT, ws)
        csw = np.imag(step(x.astype(complex), v.astype(complex), f.astype(complex), ws, ctc).x) / h
        wp, wm = np.ones(4), np.ones(4)
        wp[q] += e
        wm[q] -= e
        cp, cm = (O.CellType(m.verts, m.tris, mat, DT, w) for w in (wp, wm))
        fdw = (step(x, v, f, wp, cp).x - step(x, v, f, wm, cm).x) / (2 * e)
        assert np.max(np.abs(csw - fdw)) <= 1e-5 * np.max(np.abs(csw)), q
