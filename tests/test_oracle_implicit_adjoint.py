"""Pin of the oracle's implicit-function adjoint: the gradient of L = gx . x* + gv . v*
through the converged minimiser of a step equals central differences of a step run to
convergence, for every input kind (positions, velocities, forces, material weights), with
and without Rayleigh damping (whose dissipation term depends on x_n directly), and with
strain limits (whose projection is clamped on both sides of the deformation)."""
import numpy as np
import pytest

from oracle import npfem_oracle as O
from paper_2011_04332_b300 import inputs as I

DT = 0.1
MAT0 = (1.0, 0.05, 10.0, 10.0, 1.1)


def _converged(mat, x, v, f, mesh):
    ct = O.CellType(mesh.verts, mesh.tris, mat, DT)
    r = O.step(ct.rest, ct.solver, x, v, f, 400, tol=1e-13)
    assert r.residual < 1e-12
    return ct, r


# wrel: relative step of the weight differences.  With strain limits the energy is flat
# inside the limits, so the converged state's own rounding, divided by a 1e-6 step of the
# small bending weight, is ~2e-5 of the derivative; a 1e-4 step (no singular value lies
# within 4e-4 of a limit, so none crosses one) leaves truncation error ~1e-9.
@pytest.mark.parametrize("mesh_fn,damping,wrel", [(I.icosahedron, (), 1e-6), (lambda: I.rbc_mesh(1), (), 1e-6),
                                                  (lambda: I.rbc_mesh(1), (0.5, 1.0), 1e-6),
                                                  (lambda: I.rbc_mesh(1), (0.0, 0.0, 0.97, 1.03), 1e-4)])
def test_implicit_adjoint_matches_central_differences(mesh_fn, damping, wrel):
    MAT = MAT0 + damping
    m = mesh_fn()
    rng = np.random.default_rng(41)
    x = m.verts * np.array([1.1, 0.95, 1.0]) + 0.02 * rng.standard_normal(m.verts.shape) + 3.0
    v = 0.1 * rng.standard_normal(x.shape)
    f = 0.2 * rng.standard_normal(x.shape)
    gx_next = rng.standard_normal(x.shape)
    gv_next = 0.1 * rng.standard_normal(x.shape)
    ct, r = _converged(MAT, x, v, f, m)
    gx, gv, gf, gw = O.implicit_adjoint(ct, x, v, f, r.x, gx_next, gv_next)

    def loss(mat=None, x=x, v=v, f=f):
        mat = MAT if mat is None else mat
        _, rr = _converged(mat, x, v, f, m)
        return float(np.sum(gx_next * rr.x) + np.sum(gv_next * rr.v))

    h = 1e-6
    picks = [(int(i), int(d)) for i, d in zip(rng.integers(0, m.n, 4), rng.integers(0, 3, 4))]
    for arr, grad, name in ((x, gx, "x"), (v, gv, "v"), (f, gf, "f")):
        for i, d in picks:
            ap, am = arr.copy(), arr.copy()
            ap[i, d] += h
            am[i, d] -= h
            fd = (loss(**{name: ap}) - loss(**{name: am})) / (2 * h)
            assert grad[i, d] == pytest.approx(fd, rel=1e-5, abs=1e-7), (name, i, d)
    for q in range(4):
        mp, mm = list(MAT), list(MAT)
        hq = wrel * MAT[q]
        mp[q] += hq
        mm[q] -= hq
        fd = (loss(mat=tuple(mp)) - loss(mat=tuple(mm))) / (2 * hq)
        assert gw[q] == pytest.approx(fd, rel=1e-5, abs=1e-7), q
