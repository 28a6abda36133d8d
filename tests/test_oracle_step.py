"""Pins of the oracle's quasi-Newton time step: rest invariance, monotone objective,
the one-iteration projective-dynamics equivalence, brute-force Newton minimisation
on tiny meshes, and the history/line-search bookkeeping."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

MAT = (1.0, 0.05, 10.0, 10.0, 1.1)
DT = 0.1


def _type(mesh, mat=MAT, dt=DT, w_scale=None):
    return O.CellType(mesh.verts, mesh.tris, mat, dt, w_scale)


def test_rest_stays_at_rest():
    m = I.rbc_mesh(2)
    ct = _type(m)
    x = m.verts @ I.random_rotation(np.random.default_rng(1)).T + np.array([120.0, 40.0, 7.0])
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 5)
    assert np.max(np.abs(r.x - x)) <= 1e-14 * np.max(np.abs(x))
    assert np.max(np.abs(r.v)) <= 1e-12
    assert r.status == O.STATUS_OK


def test_free_flight_of_rigid_cell():
    """A rest-shaped cell with uniform velocity and no force translates rigidly."""
    m = I.rbc_mesh(2)
    ct = _type(m)
    v = np.tile(np.array([[0.3, -0.1, 0.2]]), (m.n, 1))
    r = O.step(ct.rest, ct.solver, m.verts, v, np.zeros_like(v), 3)
    assert np.allclose(r.x, m.verts + DT * v, rtol=0, atol=1e-13)
    assert np.allclose(r.v, v, rtol=0, atol=1e-11)


def test_uniform_gravity_like_force():
    """A uniform acceleration a (f = m a) on a rest cell: exact result x + dt^2 a."""
    m = I.rbc_mesh(2)
    ct = _type(m)
    a = np.array([0.0, 0.0, -2.0])
    f = ct.rest.mass[:, None] * a[None, :]
    r = O.step(ct.rest, ct.solver, m.verts, np.zeros_like(f), f, 2)
    assert np.allclose(r.x, m.verts + DT * DT * a, rtol=0, atol=1e-13)


def test_objective_decreases_every_iteration():
    b = I.single_rbc(seed=1000, subdiv=2, iters=8)
    m = b.types[0].mesh
    ct = _type(m)
    x, v, f = b.cell_state(0)
    f = f * 50.0   # large forces: strongly nonlinear step
    for s in range(3):
        r = O.step(ct.rest, ct.solver, x, v, f, 8)
        e = np.array(r.energies)
        assert np.all(e[1:] <= e[:-1] + 1e-6 * np.abs(e[:-1]))   # the energy guard: 1e-6 relative
        assert r.grad_norms[-1] < r.grad_norms[0]
        x, v = r.x, r.v


def test_linear_momentum_balance_at_any_iteration_count():
    """sum_i m_i v_i^{n+1} = sum_i m_i v_i^n + dt sum_i f_i after any number of iterations.
    Implicit Euler with translation-invariant energies balances momentum at its minimiser;
    the iteration keeps the balance at every iterate because it starts at the inertial
    prediction y (sum_i m_i (x_i - y_i) = 0) and A 1 = m/dt^2 makes every L-BFGS direction
    momentum-free (sum_i m_i d_i = dt^2 sum_i g_i = 0 by induction over the history).  A wrong
    mass in the inertial term or in A, or a dropped dt^2 f/m in y, breaks it."""
    for mesh, mat in ((I.rbc_mesh(2), MAT), (I.platelet_mesh(1), I.PLT_MATERIAL.as_tuple())):
        ct = _type(mesh, mat)
        m = ct.rest.mass[:, None]
        rng = np.random.default_rng(41)
        x = mesh.verts @ I.random_rotation(rng).T + rng.uniform(-50, 50, 3)
        v = 0.05 * rng.standard_normal(x.shape)
        f = 0.02 * rng.standard_normal(x.shape)
        for iters in (0, 1, 2, 5, 9):
            r = O.step(ct.rest, ct.solver, x, v, f, iters)
            p_expect = (m * v).sum(axis=0) + DT * f.sum(axis=0)
            p_got = (m * r.v).sum(axis=0)
            scale = (m * np.abs(r.v)).sum()
            assert np.max(np.abs(p_got - p_expect)) <= 1e-13 * scale, (iters, p_got - p_expect)
            assert np.max(np.abs(DT * f.sum(axis=0))) > 1e-3 * scale   # the forces' impulse counts


def _rough_start(dt, noise, seed=3):
    """A 162-vertex RBC with positions scattered by `noise` um about its rest shape: far
    from the minimiser, so that the line search has to shorten steps."""
    m = I.rbc_mesh(2)
    ct = _type(m, dt=dt)
    x = m.verts + noise * np.random.default_rng(seed).standard_normal(m.verts.shape)
    return ct, x


@pytest.mark.parametrize("dt,noise", [(0.1, 1.0), (10.0, 0.3), (1000.0, 1.0)])
def test_line_search_halves_and_never_raises_the_objective(dt, noise):
    """Backtracking from alpha = 1 by halving: every accepted step length is a power of two
    (and some are below 1 from these rough starts), and no accepted iterate raises the
    objective by more than the energy guard (1e-6 relative)."""
    ct, x = _rough_start(dt, noise)
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 8)
    a = np.array(r.alphas)
    assert np.array_equal(a, 2.0 ** np.round(np.log2(a)))
    assert a.min() < 1.0
    e = np.array(r.energies)
    assert np.all(e[1:] <= e[:-1] + 1e-6 * np.abs(e[:-1]))


def test_history_holds_the_five_newest_pairs(monkeypatch):
    """The two-loop recursion of iteration k sees min(k, 5) pairs (history 5), the newest
    last (its y the difference of the last two gradients)."""
    ct, x = _rough_start(0.1, 0.3)
    seen = []
    real = O.two_loop

    def spy(g, S, Y, solver):
        seen.append(([s.copy() for s in S], [y.copy() for y in Y], g.copy()))
        return real(g, S, Y, solver)

    monkeypatch.setattr(O, "two_loop", spy)
    iters = 9
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), iters)
    assert len(seen) == iters
    assert [len(S) for S, _, _ in seen] == [min(k, 5) for k in range(iters)]
    # the newest pair's y is the difference of the gradients the last two recursions saw
    for k in range(1, iters):
        S, Y, g = seen[k]
        assert np.array_equal(Y[-1], g - seen[k - 1][2])


@pytest.mark.parametrize("kappa,alpha", [(1.998, 1.0), (2.002, 0.5)])
def test_sufficient_decrease_on_a_one_contact_quadratic(kappa, alpha):
    """With no elastic energy and one penetrating contact on vertex i, the objective is the
    quadratic a u^2/2 + w (pen - u)^2/2 along the contact normal (a = m_i/dt^2), while the
    PD matrix holds only a: the first direction is u = w pen / a, and the full step keeps the
    fraction 1 - kappa/2 of its predicted decrease, kappa = (a + w)/a.  The weak sufficient
    decrease of the line search takes it at kappa = 1.998 (fraction 1e-3) and halves it at
    kappa = 2.002 (fraction -1e-3; at alpha = 1/2 the fraction is 1 - kappa/4): one
    iteration moves vertex i by alpha w pen / a along the normal and no other vertex."""
    m = I.icosphere(1)
    ct = _type(m, (0.0, 0.0, 0.0, 0.0, 1.1))
    i = 5
    a = ct.rest.mass[i] / DT ** 2
    n = np.array([0.6, 0.0, 0.8])
    x = m.verts + np.array([3.0, -1.0, 2.0])
    delta, depth = 0.01, 0.05
    c = n @ x[i] + depth                     # gap n.x_i - c = -depth: penetrating
    w = (kappa - 1.0) * a
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 1,
               contact=(np.array([i]), n[None, :], np.array([c]), delta, w))
    assert r.alphas == [alpha]
    assert r.x[i] - x[i] == pytest.approx(alpha * w * (delta + depth) / a * n, rel=1e-12, abs=1e-15)
    assert np.array_equal(np.delete(r.x, i, axis=0), np.delete(x, i, axis=0))


def test_collapsed_strain_only_cell_is_flagged_and_stays():
    """A strain-only cell collapsed to a point, at rest: every triangle is degenerate and
    contributes nothing, so the gradient is exactly zero; the step leaves the state where it
    is, flags the degenerate elements in its status, and reports residual 0 (|g0| = 0)."""
    m = I.rbc_mesh(1)
    ct = _type(m, (1.0, 0.0, 0.0, 0.0, 1.1))
    x = np.tile(np.array([[2.0, -1.0, 0.5]]), (m.n, 1))
    r = O.step(ct.rest, ct.solver, x, np.zeros_like(x), np.zeros_like(x), 3)
    assert np.array_equal(r.x, x)
    assert np.array_equal(r.v, np.zeros_like(x))
    assert r.status == O.STATUS_DEGENERATE
    assert r.residual == 0.0
    assert r.grad_norms == [0.0] * 4


def test_one_iteration_equals_projective_dynamics_step():
    """With no area/volume energy and one iteration, quasi-Newton PD reduces to one
    local/global PD step: x1 = A^-1 (M y/dt^2 + sum_t w_t G_t^T p_t + sum_e w_e c_e p_e)."""
    m = I.rbc_mesh(2)
    mat = (1.0, 0.05, 0.0, 0.0, 1.1)
    ct = _type(m, mat)
    rs = ct.rest
    rng = np.random.default_rng(21)
    x = m.verts
    v = 0.5 * rng.standard_normal(x.shape)
    f = 0.05 * rng.standard_normal(x.shape)
    r = O.step(rs, ct.solver, x, v, f, 1)
    assert r.alphas == [1.0]
    # independent assembly of the PD right-hand side at y
    y = x + DT * v + DT * DT * f / rs.mass[:, None]
    Fy = O.deformation_gradient(rs, y)
    P, _ = O.polar_project(Fy)
    rhs = rs.mass[:, None] * y / DT ** 2
    S = np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
    for t in range(rs.tris.shape[0]):
        G = rs.Dm_inv[t].T @ S                         # F_row^T = G [x0 x1 x2]_coord
        contrib = rs.w_tri[t] * G.T @ P[t].T           # [3 verts, 3 coords]
        np.add.at(rhs, rs.tris[t], contrib)
    K = O.hinge_K(rs, y)
    p = O.bending_project(rs, K)
    for e in range(rs.hinges.shape[0]):
        np.add.at(rhs, rs.hinges[e], rs.w_hinge[e] * np.outer(rs.c_hinge[e], p[e]))
    x1 = np.linalg.solve(O.pd_matrix(rs), rhs)
    assert np.allclose(r.x, x1, rtol=0, atol=1e-12 * np.max(np.abs(x1)))


def _newton_minimise(rs, y, x0, tol=1e-13, max_it=60):
    """Full Newton with a Hessian from central differences of the analytic gradient,
    plus backtracking; used only as an independent minimiser."""
    x = x0.copy()
    n3 = x.size
    for it in range(max_it):
        parts, g = O.objective(rs, x, y)
        if np.linalg.norm(g) < tol:
            break
        h = 1e-7
        H = np.zeros((n3, n3))
        for k in range(n3):
            e = np.zeros(n3)
            e[k] = h
            gp = O.objective(rs, x + e.reshape(x.shape), y)[1].ravel()
            gm = O.objective(rs, x - e.reshape(x.shape), y)[1].ravel()
            H[:, k] = (gp - gm) / (2 * h)
        H = 0.5 * (H + H.T)
        d = -np.linalg.solve(H, g.ravel()).reshape(x.shape)
        a = 1.0
        f0 = parts.total
        while O.objective(rs, x + a * d, y)[0].total > f0 and a > 1e-8:
            a *= 0.5
        x = x + a * d
    return x


@pytest.mark.parametrize("mesh_fn,dt", [(I.tetrahedron, 0.5), (I.icosahedron, 0.5)])
def test_lbfgs_agrees_with_brute_force_newton(mesh_fn, dt):
    """Many quasi-Newton iterations reach the exact minimiser of the step objective."""
    m = mesh_fn()
    mat = (1.0, 0.05, 10.0, 10.0, 1.1)
    ct = _type(m, mat, dt)
    rs = ct.rest
    rng = np.random.default_rng(31)
    x = m.verts
    v = 0.2 * rng.standard_normal(x.shape)
    f = 0.3 * rng.standard_normal(x.shape)
    r = O.step(rs, ct.solver, x, v, f, 200)
    ctr = x.mean(axis=0)
    y = (x - ctr) + dt * v + dt * dt * f / rs.mass[:, None]
    xs = _newton_minimise(rs, y, y.copy()) + ctr
    radius = np.max(np.linalg.norm(xs - xs.mean(axis=0), axis=1))
    assert np.max(np.abs(r.x - xs)) <= 1e-10 * radius
    assert r.residual < 1e-10


def test_history_is_bounded_and_curvature_checked():
    g = np.random.default_rng(1).standard_normal((10, 3))
    A = np.diag(np.arange(1, 11, dtype=float))
    gs = O.GlobalSolver(A)
    # with no history the two-loop is exactly H0 g = A^-1 g
    assert np.allclose(O.two_loop(g, [], [], gs), np.linalg.solve(A, g))
    # secant condition: with one pair (s, y), H y = s
    s = np.random.default_rng(2).standard_normal((10, 3))
    y = np.random.default_rng(3).standard_normal((10, 3))
    y = y + 5 * s                    # make s.y > 0
    assert np.allclose(O.two_loop(y, [s], [y], gs), s)


def test_two_loop_equals_dense_bfgs_inverse_update():
    """With several pairs the two-loop recursion is the BFGS inverse-Hessian update
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T applied oldest -> newest from
    H0 = A^-1 (per coordinate), written out densely over the 3n components; the newest
    pair also satisfies the secant condition H y = s exactly."""
    rng = np.random.default_rng(7)
    n = 9
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    gs = O.GlobalSolver(A)
    S, Y = [], []
    for _ in range(4):
        s = rng.standard_normal((n, 3))
        y = rng.standard_normal((n, 3)) + 3 * s
        assert np.sum(s * y) > 0
        S.append(s)
        Y.append(y)
    H = np.kron(np.linalg.inv(A), np.eye(3))      # flat index 3 i + c of an (n, 3) array
    I3n = np.eye(3 * n)
    for s, y in zip(S, Y):
        sf, yf = s.ravel(), y.ravel()
        rho = 1.0 / (sf @ yf)
        V = I3n - rho * np.outer(yf, sf)
        H = V.T @ H @ V + rho * np.outer(sf, sf)
    g = rng.standard_normal((n, 3))
    r = O.two_loop(g, S, Y, gs)
    assert np.allclose(r.ravel(), H @ g.ravel(), rtol=1e-12, atol=1e-12 * np.max(np.abs(r)))
    assert np.allclose(O.two_loop(Y[-1], S, Y, gs), S[-1], rtol=1e-12, atol=1e-12)
    # the order matters: the reversed history is a different operator
    assert not np.allclose(O.two_loop(g, S[::-1], Y[::-1], gs), r, rtol=1e-6)


def test_complex_step_derivative_matches_central_differences():
    """The oracle's forward-mode derivative (complex step through the whole step,
    forces and weight scales) agrees with central differences of the real step."""
    m = I.rbc_mesh(1)
    b = I.single_rbc(subdiv=1)
    ct = _type(m)
    x, v, f = b.cell_state(0)
    f = 30 * f
    rng = np.random.default_rng(0)
    df = rng.standard_normal(f.shape) * 1e-3
    h = 1e-30
    rc = O.step(ct.rest, ct.solver, x.astype(complex), v.astype(complex), f + 1j * h * df, 5)
    cs = np.imag(rc.x) / h
    e = 1e-4
    fd = (O.step(ct.rest, ct.solver, x, v, f + e * df, 5).x - O.step(ct.rest, ct.solver, x, v, f - e * df, 5).x) / (2 * e)
    assert np.max(np.abs(cs - fd)) <= 1e-6 * np.max(np.abs(cs))
    for q in range(4):
        ws = np.ones(4, complex)
        ws[q] += 1j * h
        ctc = _type(m, w_scale=ws)
        csw = np.imag(O.step(ctc.rest, ctc.solver, x.astype(complex), v.astype(complex), f.astype(complex), 5, ws).x) / h
        e = 1e-5
        wp, wm = np.ones(4), np.ones(4)
        wp[q] += e
        wm[q] -= e
        cp, cm = _type(m, w_scale=wp), _type(m, w_scale=wm)
        fdw = (O.step(cp.rest, cp.solver, x, v, f, 5, wp).x - O.step(cm.rest, cm.solver, x, v, f, 5, wm).x) / (2 * e)
        assert np.max(np.abs(csw - fdw)) <= 2e-5 * np.max(np.abs(csw)), q


def test_converged_residual_mode_stops_at_first_iterate_below_tol():
    """Converged-residual mode: the step ends after the first iteration whose
    gradient norm falls below tol |g0|; that run equals a fixed-budget run of the
    same length, every shorter run is still above tol, and the stopped iterate
    lies within the tolerance's reach of the exact minimiser (brute-force Newton)."""
    m = I.icosahedron()
    dt = 0.5
    ct = _type(m, MAT, dt)
    rs = ct.rest
    rng = np.random.default_rng(31)
    x = m.verts
    v = 0.2 * rng.standard_normal(x.shape)
    f = 0.3 * rng.standard_normal(x.shape)
    ctr = x.mean(axis=0)
    y = (x - ctr) + dt * v + dt * dt * f / rs.mass[:, None]
    xs = _newton_minimise(rs, y, y.copy()) + ctr
    radius = np.max(np.linalg.norm(xs - xs.mean(axis=0), axis=1))
    prev = 0
    for tol in (1e-2, 1e-4, 1e-6, 1e-9):
        r = O.step(rs, ct.solver, x, v, f, 200, tol=tol)
        k = len(r.alphas)
        assert r.residual < tol and k < 200 and k >= prev
        assert all(gn >= tol * r.grad_norms[0] for gn in r.grad_norms[:-1])
        fixed = O.step(rs, ct.solver, x, v, f, k)
        assert np.array_equal(fixed.x, r.x) and np.array_equal(fixed.v, r.v)
        if k > 1:
            assert O.step(rs, ct.solver, x, v, f, k - 1).residual >= tol
        prev = k
    assert np.max(np.abs(r.x - xs)) <= 1e-7 * radius


def test_converged_residual_mode_zero_gradient_runs_budget():
    """A cell already at the minimiser (|g0| = 0) never meets |g| < tol |g0| and so
    runs its whole budget; its state is unchanged."""
    m = I.rbc_mesh(1)
    ct = _type(m)
    r = O.step(ct.rest, ct.solver, m.verts, np.zeros_like(m.verts), np.zeros_like(m.verts),
               4, tol=1e-3)
    assert len(r.alphas) == 4
    assert np.max(np.abs(r.x - m.verts)) <= 1e-14 * np.max(np.abs(m.verts))
