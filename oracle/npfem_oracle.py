"""Plain CPU FP64 oracle of one npFEM time step for closed triangulated membranes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module; only tests/, the smoke check and the benchmark's CPU-baseline leg do.
It shares no code with the CUDA path (the only shared module is the seeded
input generator, which holds none of the method's arithmetic).

What it computes, and where each piece comes from
-------------------------------------------------
* The solid is solved by npFEM, a mass-lumped linear finite-element solver on
  triangulated membranes, implicit in time (Introduction; Implementation and
  architecture).  It discretises the elastodynamics equation, Eq. (2).
* npFEM is derived from ShapeOp / projective dynamics (Bouaziz et al. 2014) and
  advances bodies with the quasi-Newton projective-dynamics kernel of Liu et
  al. 2017 (Implementation and architecture, first bullet), iterated towards a
  converged solution rather than a fixed graphics budget (second bullet).
* The material is a sum of per-element energies, each with a weight and
  parameters (Setting up new materials section).
* Per step the solid solver receives external forces and returns positions and
  velocities (Implementation and architecture).
* Viscoelastic damping (optional): the bodies' viscous behaviour is set by two
  parameters, Calpha and Cbeta (Setting up new materials section), read here as
  Rayleigh damping C = Calpha M + Cbeta L (L the elastic part of the PD matrix) in
  implicit Euler: a dissipation term in the objective and C/dt in the matrix.
* Strain limits (optional): the membrane-strain constraint set of a triangle is the set
  of deformation gradients whose singular values lie in [s_min, s_max] (ShapeOp-style
  strain limiting, the solver's origin named in the Implementation and architecture
  section; per-material parameters, Setting up new materials section); the default
  [1, 1] is the set of rotations.
* Collisions (optional): contact detection at the start of a step and a penalty
  per contact in the step objective; the paper names collision detection and
  collision forces (Performance figure, "Other"), a collision weight (Collision at
  an obstacle section) and a fluid-free cell-packing application (Cell Packing
  section), without formulas: the reading is stated at `detect_contacts`.

The paper prints no formulas for the energies or the iteration; the readings
used here (strain = distance of the triangle deformation gradient to the
rotations, cotangent hinge bending with rest-curvature magnitude, quadratic
global area/volume penalties, Armijo line search with an approximate-Armijo
fallback, history 5) are listed with their reasons in the project design notes.

Parity pins: every function here is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute-force Newton minimisation and finite
differences (no function is "parity unpinned").

Implementation style: plain numpy float64, vectorised over elements only.  A
dense Cholesky from numpy serves as the library step for the global matrix.
Every function also accepts complex inputs with an infinitesimal imaginary part
(complex-step differentiation): norms are written as sqrt(sum(x*x)), decisions use
real parts, and the global solve propagates an imaginary perturbation of A or of
the right-hand side exactly to first order.  This gives the oracle its own
forward-mode derivative, used to check the CUDA adjoint.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

# Line-search / history constants (readings; identical on the CUDA side).
ARMIJO_C1 = 1e-4
MAX_HALVINGS = 20
ENERGY_GUARD_EPS = 1e-6        # approximate-Armijo energy guard, relative
CURVATURE_EPS = 1e-12          # skip pair when s.y <= eps*|s||y|
HISTORY = 5
DEGENERATE_DET = 1e-30         # det(F^T F) below this: element contributes nothing
DEGENERATE_NORM = 1e-30        # |K| below this: projection falls back to K0

STATUS_OK = 0
STATUS_LINESEARCH_FAIL = 1
STATUS_DEGENERATE = 2
STATUS_NONFINITE = 4


# ---------------------------------------------------------------- topology
def hinges_of(tris: np.ndarray, n: int) -> np.ndarray:
    """Interior edges of a closed oriented mesh as hinges [E, 4] = (i, j, kA, kB).

    (i, j) is the shared edge with i < j; kA is the vertex opposite the edge in
    the triangle that traverses i -> j, kB the one in the triangle traversing
    j -> i.  Raises ValueError when the mesh is not a closed 2-manifold.
    """
    directed = {}
    for t in tris:
        for a, b, c in ((t[0], t[1], t[2]), (t[1], t[2], t[0]), (t[2], t[0], t[1])):
            key = (int(a), int(b))
            if key in directed:
                raise ValueError("edge traversed twice in the same direction")
            directed[key] = int(c)
    hinges = []
    for (a, b), c in directed.items():
        if a < b:
            if (b, a) not in directed:
                raise ValueError("open edge: mesh is not closed")
            hinges.append((a, b, c, directed[(b, a)]))
    hinges.sort()
    return np.array(hinges, dtype=np.int64).reshape(-1, 4)


# ---------------------------------------------------------------- rest state
@dataclasses.dataclass
class RestState:
    """Per-cell-type constants computed once from the rest mesh (setup step)."""
    n: int
    tris: np.ndarray        # [T, 3]
    hinges: np.ndarray      # [E, 4]
    Dm_inv: np.ndarray      # [T, 2, 2] inverse rest edge matrix in the local frame
    area_rest: np.ndarray   # [T]
    w_tri: np.ndarray       # [T]   strain weight per triangle = w_strain * rest area
    c_hinge: np.ndarray     # [E, 4] cotangent hinge stencil
    kappa0: np.ndarray      # [E]   rest |K|
    K0: np.ndarray          # [E, 3] rest K (tie-break direction)
    w_hinge: np.ndarray     # [E]   bending weight per hinge = w_bend * 3/(A_A + A_B)
    A0: float
    V0: float
    mass: np.ndarray        # [n] lumped nodal masses
    w_area: float
    w_vol: float
    dt: float
    c_alpha: float = 0.0    # Rayleigh damping: C = c_alpha M + c_beta L (1/us, us)
    c_beta: float = 0.0
    s_min: float = 1.0      # strain limits: singular values of F clamped to [s_min, s_max]
    s_max: float = 1.0


def _cot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Cotangent of the angle between row vectors a and b."""
    return np.einsum("ij,ij->i", a, b) / np.linalg.norm(np.cross(a, b), axis=1)


def rest_state(X: np.ndarray, tris: np.ndarray, w_strain: float, w_bend: float,
               w_area: float, w_vol: float, density: float, dt: float,
               c_alpha: float = 0.0, c_beta: float = 0.0, s_min: float = 1.0, s_max: float = 1.0) -> RestState:
    """Rest-shape constants of a cell type (mass-lumped linear FE, Introduction).

    * Each triangle gets a local orthonormal frame (u along the first edge, w in
      the plane) and Dm = [e1 e2] expressed in it; F = [x1-x0, x2-x0] Dm^-1.
    * Each interior edge gets the cotangent hinge stencil c (sums to zero and
      annihilates flat hinges) and its rest magnitude |K0|.
    * Lumped masses: the cell mass density*V0 is spread by the area share of
      each vertex (a third of the incident rest triangle areas).
    """
    if not (0.0 < s_min <= 1.0 <= s_max < np.inf):
        raise ValueError("strain limits must satisfy 0 < s_min <= 1 <= s_max (the rest shape is in the set)")
    X = np.asarray(X, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    n = X.shape[0]
    x0, x1, x2 = X[tris[:, 0]], X[tris[:, 1]], X[tris[:, 2]]
    e1, e2 = x1 - x0, x2 - x0
    cr = np.cross(e1, e2)
    crn = np.linalg.norm(cr, axis=1)
    if np.any(crn <= 0):
        raise ValueError("degenerate rest triangle")
    area = 0.5 * crn
    l1 = np.linalg.norm(e1, axis=1)
    u = e1 / l1[:, None]
    nrm = cr / crn[:, None]
    w = np.cross(nrm, u)
    Dm = np.zeros((tris.shape[0], 2, 2))
    Dm[:, 0, 0] = l1
    Dm[:, 0, 1] = np.einsum("ij,ij->i", e2, u)
    Dm[:, 1, 0] = 0.0
    Dm[:, 1, 1] = np.einsum("ij,ij->i", e2, w)
    Dm_inv = np.linalg.inv(Dm)

    H = hinges_of(tris, n)
    if H.shape[0] * 2 != 3 * tris.shape[0]:
        raise ValueError("mesh is not a closed manifold")
    p0, p1, p2, p3 = X[H[:, 0]], X[H[:, 1]], X[H[:, 2]], X[H[:, 3]]
    cotA0 = _cot(p1 - p0, p2 - p0)
    cotA1 = _cot(p0 - p1, p2 - p1)
    cotB0 = _cot(p1 - p0, p3 - p0)
    cotB1 = _cot(p0 - p1, p3 - p1)
    c = np.stack([cotA1 + cotB1, cotA0 + cotB0, -(cotA0 + cotA1), -(cotB0 + cotB1)], axis=1)
    K0 = (c[:, 0, None] * p0 + c[:, 1, None] * p1 + c[:, 2, None] * p2 + c[:, 3, None] * p3)
    kappa0 = np.linalg.norm(K0, axis=1)
    areaA = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    areaB = 0.5 * np.linalg.norm(np.cross(p1 - p0, p3 - p0), axis=1)
    w_h = w_bend * 3.0 / (areaA + areaB)

    A0 = float(np.sum(area))
    ctr = X.mean(axis=0)
    V0 = float(_volume(X - ctr, tris))
    vert_area = np.zeros(n)
    for k in range(3):
        np.add.at(vert_area, tris[:, k], area / 3.0)
    mass = density * V0 * vert_area / A0
    return RestState(n, tris, H, Dm_inv, area, w_strain * area, c, kappa0, K0, w_h,
                     A0, V0, mass, float(w_area), float(w_vol), float(dt), float(c_alpha), float(c_beta),
                     float(s_min), float(s_max))


def _norm_rows(a: np.ndarray) -> np.ndarray:
    """Row norms sqrt(sum a^2), analytic for complex-step inputs."""
    return np.sqrt(np.sum(a * a, axis=1))


def _volume(x: np.ndarray, tris: np.ndarray) -> float:
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    return np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0


# ---------------------------------------------------------------- projections
def polar_project(F: np.ndarray) -> (np.ndarray, np.ndarray):
    """Closest rotation-like 3x2 matrix R = F (F^T F)^(-1/2) for a batch of F [T,3,2].

    Uses the closed form of the 2x2 SPD square root:
    sqrt(C) = (C + sqrt(det C) I) / sqrt(tr C + 2 sqrt(det C)).
    Returns (R, degenerate_mask); degenerate elements (det C <= 1e-30) get R = F.
    """
    C = np.einsum("tki,tkj->tij", F, F)
    det = C[:, 0, 0] * C[:, 1, 1] - C[:, 0, 1] * C[:, 1, 0]
    bad = np.real(det) <= DEGENERATE_DET
    det_s = np.where(bad, 1.0, det)
    s = np.sqrt(det_s)
    tau = np.sqrt(C[:, 0, 0] + C[:, 1, 1] + 2.0 * s)
    S = (C + s[:, None, None] * np.eye(2)[None]) / tau[:, None, None]
    detS = S[:, 0, 0] * S[:, 1, 1] - S[:, 0, 1] * S[:, 1, 0]
    Sinv = np.empty_like(S)
    Sinv[:, 0, 0] = S[:, 1, 1] / detS
    Sinv[:, 1, 1] = S[:, 0, 0] / detS
    Sinv[:, 0, 1] = -S[:, 0, 1] / detS
    Sinv[:, 1, 0] = -S[:, 1, 0] / detS
    R = np.einsum("tij,tjk->tik", F, Sinv)
    R[bad] = F[bad]
    return R, bad


def clamped_project(F: np.ndarray, s_min: float, s_max: float) -> (np.ndarray, np.ndarray):
    """Closest 3x2 matrix to F whose singular values lie in [s_min, s_max], for a batch
    F [T,3,2]: U clamp(Sigma) V^T (strain-limit reading of the membrane-strain
    constraint set, Setting up new materials section; [1, 1] gives the rotations).

    With C = F^T F = V Sigma^2 V^T the projection is F V diag(k_i) V^T, k_i =
    clamp(sigma_i)/sigma_i, and V diag(k1, k2) V^T = k2 I + (k1 - k2)/(l1 - l2) (C - l2 I)
    with l1 >= l2 the eigenvalues of C (the spectral projector of the 2x2 C in closed
    form); equal eigenvalues give k1 = k2 and the matrix k2 I.  Clamping decisions use
    real parts (complex-step inputs).  Returns (P, degenerate_mask); degenerate elements
    (det C <= 1e-30) get P = F, as in polar_project."""
    C = np.einsum("tki,tkj->tij", F, F)
    det = C[:, 0, 0] * C[:, 1, 1] - C[:, 0, 1] * C[:, 1, 0]
    bad = np.real(det) <= DEGENERATE_DET
    h = 0.5 * (C[:, 0, 0] + C[:, 1, 1])
    q = 0.5 * (C[:, 0, 0] - C[:, 1, 1])
    disc = np.sqrt(q * q + C[:, 0, 1] * C[:, 1, 0])
    l1 = h + disc
    # the smaller eigenvalue as det C / l1 with det C = |F0 x F1|^2 (Lagrange identity):
    # h - disc and C00 C11 - C01^2 both cancel for thin triangles
    fx = np.cross(F[:, :, 0], F[:, :, 1])
    l2 = np.where(bad, 1.0, np.sum(fx * fx, axis=1) / np.where(bad, 1.0, l1))
    sig1, sig2 = np.sqrt(l1), np.sqrt(l2)

    def k_of(sig):
        r = np.real(sig)
        return np.where(r > s_max, s_max / sig, np.where(r < s_min, s_min / sig, np.ones_like(sig)))

    k1, k2 = k_of(sig1), k_of(sig2)
    split = np.real(disc) > 0.0
    coef = np.where(split, (k1 - k2) / np.where(split, 2.0 * disc, 1.0), 0.0)   # l1 - l2 = 2 disc exactly
    eye = np.eye(2)[None]
    M = k2[:, None, None] * eye + coef[:, None, None] * (C - l2[:, None, None] * eye)
    P = np.einsum("tij,tjk->tik", F, M)
    P[bad] = F[bad]
    return P, bad


def strain_project(F: np.ndarray, s_min: float = 1.0, s_max: float = 1.0) -> (np.ndarray, np.ndarray):
    """Projection of each F onto the membrane-strain constraint set: the rotations
    (polar_project) for the default limits [1, 1], else clamped_project."""
    if s_min == 1.0 and s_max == 1.0:
        return polar_project(F)
    return clamped_project(F, s_min, s_max)


def deformation_gradient(rs: RestState, x: np.ndarray) -> np.ndarray:
    t = rs.tris
    E = np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]]], axis=2)  # [T,3,2]
    return np.einsum("tij,tjk->tik", E, rs.Dm_inv)


def hinge_K(rs: RestState, x: np.ndarray) -> np.ndarray:
    """K = sum_j c_j x_j, evaluated on edge vectors (sum c_j = 0)."""
    H, c = rs.hinges, rs.c_hinge
    base = x[H[:, 0]]
    return (c[:, 1, None] * (x[H[:, 1]] - base) + c[:, 2, None] * (x[H[:, 2]] - base)
            + c[:, 3, None] * (x[H[:, 3]] - base))


def bending_project(rs: RestState, K: np.ndarray) -> np.ndarray:
    """Closest point of K on the sphere |p| = |K0|; tie-break p = K0 for |K| ~ 0."""
    kn = _norm_rows(K)
    small = np.real(kn) < DEGENERATE_NORM
    p = rs.kappa0[:, None] * K / np.where(small, 1.0, kn)[:, None]
    p[small] = rs.K0[small]
    return p


# ---------------------------------------------------------------- objective
@dataclasses.dataclass
class EnergyParts:
    inertia: float
    strain: float
    bend: float
    area: float
    volume: float
    A: float
    V: float
    degenerate: int
    contact: float = 0.0
    damping: float = 0.0

    @property
    def total(self) -> float:
        return self.inertia + self.strain + self.bend + self.area + self.volume + self.contact + self.damping


def internal_energy_and_gradient(rs: RestState, x: np.ndarray, w_scale=None):
    """Elastic energy sum_t E_t + sum_e E_e + E_A + E_V and its gradient [n,3].

    E_t = w_t/2 |F - R(F)|^2,  grad_F = w_t (F - R)   (R: projection onto the strain
          constraint set, the rotations unless the rest state carries strain limits)
    E_e = w_e/2 |K - p(K)|^2,  grad_xj = c_j w_e (K - p)
    E_A = w_A/2 (A - A0)^2 / A0,  E_V = w_V/2 (V - V0)^2 / V0
    `w_scale` optionally multiplies (w_strain, w_bend, w_area, w_vol).
    """
    ws = np.ones(4) if w_scale is None else np.asarray(w_scale)
    n = rs.n
    g = np.zeros((n, 3), dtype=np.result_type(x, ws))
    t = rs.tris
    # --- membrane strain, per triangle
    F = deformation_gradient(rs, x)
    R, bad = strain_project(F, rs.s_min, rs.s_max)
    wt = rs.w_tri * ws[0]
    Dlt = F - R
    e_strain = 0.5 * np.sum(wt * np.einsum("tij,tij->t", Dlt, Dlt))
    P = wt[:, None, None] * Dlt                       # dE/dF  [T,3,2]
    dE = np.einsum("tij,tkj->tik", P, rs.Dm_inv)      # dE/d[e1 e2] = P Dm^-T  [T,3,2]
    np.add.at(g, t[:, 1], dE[:, :, 0])
    np.add.at(g, t[:, 2], dE[:, :, 1])
    np.add.at(g, t[:, 0], -dE[:, :, 0] - dE[:, :, 1])
    # --- bending, per hinge
    K = hinge_K(rs, x)
    p = bending_project(rs, K)
    we = rs.w_hinge * ws[1]
    r = K - p
    e_bend = 0.5 * np.sum(we * np.einsum("ij,ij->i", r, r))
    wr = we[:, None] * r
    for k in range(4):
        np.add.at(g, rs.hinges[:, k], rs.c_hinge[:, k, None] * wr)
    # --- global area
    a, b, c = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    cr = np.cross(b - a, c - a)
    crn = _norm_rows(cr)
    A = 0.5 * np.sum(crn)
    nh = cr / np.where(np.real(crn) > 0, crn, 1.0)[:, None]
    kA = ws[2] * rs.w_area * (A - rs.A0) / rs.A0
    e_area = 0.5 * ws[2] * rs.w_area * (A - rs.A0) ** 2 / rs.A0
    np.add.at(g, t[:, 0], kA * 0.5 * np.cross(nh, c - b))
    np.add.at(g, t[:, 1], kA * 0.5 * np.cross(nh, a - c))
    np.add.at(g, t[:, 2], kA * 0.5 * np.cross(nh, b - a))
    # --- global volume (about the centroid, translation invariant on a closed mesh)
    ctr = x.mean(axis=0)
    aa, bb, cc = a - ctr, b - ctr, c - ctr
    V = np.sum(np.einsum("ij,ij->i", aa, np.cross(bb, cc))) / 6.0
    kV = ws[3] * rs.w_vol * (V - rs.V0) / rs.V0
    e_vol = 0.5 * ws[3] * rs.w_vol * (V - rs.V0) ** 2 / rs.V0
    np.add.at(g, t[:, 0], kV * np.cross(bb, cc) / 6.0)
    np.add.at(g, t[:, 1], kV * np.cross(cc, aa) / 6.0)
    np.add.at(g, t[:, 2], kV * np.cross(aa, bb) / 6.0)
    parts = EnergyParts(0.0, e_strain, e_bend, e_area, e_vol, A, V, int(np.sum(bad)))
    return parts, g


def objective(rs: RestState, x: np.ndarray, y: np.ndarray, w_scale=None, contact=None, damp=None, walls=None):
    """Implicit-Euler variational objective of one step (Eq. (2) discretised):
    f(x) = (x-y)^T M (x-y) / (2 dt^2) + E_int(x) [+ E_contact(x)] [+ E_damp(x)], and its
    gradient.  contact: (idx, nrm, crel, delta, weight) as in contact_energy_and_gradient.
    walls: (lo, hi, delta, weight) in the coordinates of x, as in wall_energy_and_gradient.
    damp: (x_n, C) with the step's start x_n and C = damping_matrix: the dissipation term
    E_damp = (x - x_n)^T C (x - x_n) / (2 dt) per coordinate joins; the stationarity
    condition is then implicit Euler for M a + C v + grad E = f."""
    parts, g = internal_energy_and_gradient(rs, x, w_scale)
    dx = x - y
    m = rs.mass
    parts.inertia = np.sum(m[:, None] * dx * dx) / (2.0 * rs.dt ** 2)
    g = g + m[:, None] * dx / rs.dt ** 2
    if damp is not None:
        x_n, C = damp
        u = x - x_n
        Cu = C @ u
        parts.damping = np.sum(u * Cu) / (2.0 * rs.dt)
        g = g + Cu / rs.dt
    if contact is not None:
        ec, gc = contact_energy_and_gradient(x, *contact)
        parts.contact = ec
        g = g + gc
    if walls is not None:
        ew, gw = wall_energy_and_gradient(x, *walls)
        parts.contact = parts.contact + ew
        g = g + gw
    return parts, g


# ---------------------------------------------------------------- contacts
# Collision reading (the paper names collision detection, collision forces and a
# collision weight, and a fluid-free cell-packing application in which npFEM resolves
# the overlaps of randomly placed cells: Performance figure, Cell Packing and
# Collision at an obstacle sections; it gives no formula).  At the start of a step,
# every vertex i of cell a is matched with the nearest vertex j of each other cell b
# within a search radius; the two nearest such cells are kept.  Each kept match is a
# plane through x_j with normal n_j, the unit area-weighted outward vertex normal of
# b at j, both from the step's input state and fixed during the step.  The step
# objective gains, per kept match, the one-sided quadratic penalty
#     E = (w/2) max(0, delta - (n_j . x_i - n_j . x_j))^2,
# delta a contact thickness, w the collision weight: a ShapeOp-style energy outside
# the prefactored matrix (like the area and volume terms), so cells stay independent
# within a step.
CONTACT_SLOTS = 2


def vertex_normals(x: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Unit area-weighted outward vertex normals [n,3]: the sum over incident
    triangles, in triangle order, of (x1 - x0) x (x2 - x0), normalised."""
    N = np.cross(x[tris[:, 1]] - x[tris[:, 0]], x[tris[:, 2]] - x[tris[:, 0]])
    acc = np.zeros_like(x)
    np.add.at(acc, tris.reshape(-1), np.repeat(N, 3, axis=0))
    return acc / _norm_rows(acc)[:, None]


def _sq_dist(x: np.ndarray, i: int) -> np.ndarray:
    """|x_i - x_j|^2 for every column j of x [3,N], evaluated as (dx*dx + dy*dy) + dz*dz."""
    dx = x[0, i] - x[0]
    dy = x[1, i] - x[1]
    dz = x[2, i] - x[2]
    return (dx * dx + dy * dy) + dz * dz


def vertex_contacts(x: np.ndarray, offsets, cell_of_vertex: np.ndarray, i: int, radius: float,
                    index=None):
    """The matches of global vertex i: a list of (d2, b, j), nearest cell first, at
    most CONTACT_SLOTS.  Per other cell b the vertex j of b nearest to x_i (equal
    distances: the smaller j); cells with that distance below `radius` compete, and
    equal distances go to the smaller b."""
    a = int(cell_of_vertex[i])
    # |x_i - x_j| < radius needs |dx| < radius: only those columns can match (and they
    # hold every vertex of a cell that is at least as near as that cell's match).  With
    # `index` = (argsort of x[0], sorted x[0]) the columns come from a window 1 % wider.
    if index is None:
        cand = np.nonzero(np.abs(x[0] - x[0, i]) < radius)[0]
    else:
        order, xs = index
        lo = np.searchsorted(xs, x[0, i] - 1.01 * radius, side="left")
        hi = np.searchsorted(xs, x[0, i] + 1.01 * radius, side="right")
        cand = np.sort(order[lo:hi])
    d2 = _sq_dist(x[:, cand], int(np.searchsorted(cand, i))) if len(cand) else np.zeros(0)
    r2 = radius * radius
    found = []
    for b in np.unique(cell_of_vertex[cand[d2 < r2]]):
        b = int(b)
        if b == a:
            continue
        inb = np.nonzero(cell_of_vertex[cand] == b)[0]    # b's candidates, increasing j
        k = int(np.argmin(d2[inb]))                      # first occurrence: the smaller j on ties
        found.append((float(d2[inb][k]), b, int(cand[inb[k]])))
    found.sort(key=lambda t: (t[0], t[1]))
    return found[:CONTACT_SLOTS]


def detect_contacts(types: List["CellType"], type_of_cell, offsets, x: np.ndarray, radius: float,
                    vertices=None) -> Dict[str, np.ndarray]:
    """Contacts of the step's input state x [3,N] (brute force over all vertices):
    per vertex the count (0..2), the matched vertex j and cell b per slot, and the
    plane of each slot: unit normal n_j [3] and offset c = n_j . x_j (absolute
    coordinates).  Unused slots hold j = b = -1 and zeros.  `vertices` restricts the
    search to those global vertices (the others report no contact)."""
    N = x.shape[1]
    ncells = len(type_of_cell)
    cell_of_vertex = np.repeat(np.arange(ncells), np.diff(np.asarray(offsets)))
    cnt = np.zeros(N, dtype=np.int32)
    jj = np.full((N, CONTACT_SLOTS), -1, dtype=np.int64)
    bb = np.full((N, CONTACT_SLOTS), -1, dtype=np.int64)
    nrm = np.zeros((N, CONTACT_SLOTS, 3))
    cc = np.zeros((N, CONTACT_SLOTS))
    normals = {}
    order = np.argsort(x[0], kind="stable")
    index = (order, x[0][order])
    for i in (range(N) if vertices is None else vertices):
        for k, (_, b, j) in enumerate(vertex_contacts(x, offsets, cell_of_vertex, i, radius, index)):
            if b not in normals:
                s = slice(int(offsets[b]), int(offsets[b + 1]))
                normals[b] = vertex_normals(x[:, s].T, types[int(type_of_cell[b])].rest.tris)
            nj = normals[b][j - int(offsets[b])]
            cnt[i] = k + 1
            jj[i, k], bb[i, k] = j, b
            nrm[i, k] = nj
            cc[i, k] = float(np.sum(nj * x[:, j]))
    return {"count": cnt, "vertex": jj, "cell": bb, "normal": nrm, "offset": cc}


def cell_contacts(contacts: Dict[str, np.ndarray], o0: int, o1: int):
    """The matches of the vertices [o0, o1) as flat arrays (local vertex index,
    normal [m,3], absolute plane offset [m]), in vertex order then slot order."""
    idx, nrm, off = [], [], []
    for i in range(o0, o1):
        for k in range(int(contacts["count"][i])):
            idx.append(i - o0)
            nrm.append(contacts["normal"][i, k])
            off.append(contacts["offset"][i, k])
    return (np.array(idx, dtype=np.int64), np.array(nrm).reshape(-1, 3), np.array(off))


def wall_energy_and_gradient(x: np.ndarray, lo: np.ndarray, hi: np.ndarray, delta: float, weight: float):
    """Box walls (cell-wall contact of the collision reading): the faces of the box
    [lo, hi] act on every vertex with the contacts' one-sided penalty,
    E = sum_v sum_d (w/2) [max(0, delta - (x_vd - lo_d))^2 + max(0, delta - (hi_d - x_vd))^2],
    with lo, hi in the coordinates of x.  Returns E and the gradient [n,3]."""
    pl = delta - (x - lo[None, :])
    pl = np.where(np.real(pl) > 0.0, pl, 0.0)
    ph = delta - (hi[None, :] - x)
    ph = np.where(np.real(ph) > 0.0, ph, 0.0)
    E = 0.5 * weight * (np.sum(pl * pl) + np.sum(ph * ph))
    return E, weight * (ph - pl)


def contact_energy_and_gradient(x: np.ndarray, idx: np.ndarray, nrm: np.ndarray, crel: np.ndarray,
                                delta: float, weight: float):
    """E = sum_k (w/2) max(0, delta - (n_k . x_idx[k] - crel_k))^2 and its gradient
    [n,3] (-w max(0, .) n_k on vertex idx[k]); crel is the plane offset in the
    coordinates of x."""
    g = np.zeros_like(x)
    if len(idx) == 0:
        return 0.0, g
    gap = np.sum(nrm * x[idx], axis=1) - crel
    pen = delta - gap
    pen = np.where(np.real(pen) > 0.0, pen, 0.0)
    E = 0.5 * weight * np.sum(pen * pen)
    np.add.at(g, idx, -weight * pen[:, None] * nrm)
    return E, g


# ---------------------------------------------------------------- global matrix
def elastic_matrix(rs: RestState, w_scale=None) -> np.ndarray:
    """The elastic part of the projective-dynamics matrix (n x n, shared by x, y, z):
    L = sum_t w_t G_t^T G_t + sum_e w_e c_e c_e^T, where G_t maps a triangle's three
    vertex coordinates to one row of F."""
    ws = np.ones(4) if w_scale is None else np.asarray(w_scale)
    n = rs.n
    A = np.zeros((n, n), dtype=np.result_type(ws, np.float64))
    S = np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
    for ti in range(rs.tris.shape[0]):
        G = rs.Dm_inv[ti].T @ S                    # [2,3]
        blk = ws[0] * rs.w_tri[ti] * (G.T @ G)
        idx = rs.tris[ti]
        A[np.ix_(idx, idx)] += blk
    for e in range(rs.hinges.shape[0]):
        cvec = rs.c_hinge[e]
        idx = rs.hinges[e]
        A[np.ix_(idx, idx)] += ws[1] * rs.w_hinge[e] * np.outer(cvec, cvec)
    return A


def damping_matrix(rs: RestState, w_scale=None) -> np.ndarray:
    """Rayleigh damping C = c_alpha M + c_beta L (damping reading: viscous behaviour of
    the bodies set by Calpha and Cbeta, Setting up new materials section)."""
    return rs.c_alpha * np.diag(rs.mass) + rs.c_beta * elastic_matrix(rs, w_scale)


def pd_matrix(rs: RestState, w_scale=None) -> np.ndarray:
    """Projective-dynamics system matrix (n x n, shared by x, y, z):
    A = M/dt^2 + L, plus C/dt with Rayleigh damping, i.e.
    A = (1/dt^2 + c_alpha/dt) M + (1 + c_beta/dt) L  (L: elastic_matrix)."""
    dt = rs.dt
    L = elastic_matrix(rs, w_scale)
    return np.diag(rs.mass * (1.0 / dt ** 2 + rs.c_alpha / dt)) + (1.0 + rs.c_beta / dt) * L


class GlobalSolver:
    """H0 = A^-1 applied coordinate-wise through a dense Cholesky factor A = L L^T.

    For a complex-step matrix A = Ar + i Ai (Ai infinitesimal) and right-hand side
    q = qr + i qi, the solution is zr = Ar^-1 qr, zi = Ar^-1 (qi - Ai zr), exact to
    first order in the imaginary parts."""

    def __init__(self, A: np.ndarray):
        self.A = A
        self.Ai = np.imag(A) if np.iscomplexobj(A) else None
        self.L = np.linalg.cholesky(np.real(A))

    def _real_solve(self, q):
        import scipy.linalg as sla
        z = sla.solve_triangular(self.L, q, lower=True)
        return sla.solve_triangular(self.L.T, z, lower=False)

    def solve(self, q: np.ndarray) -> np.ndarray:
        if not np.iscomplexobj(q) and self.Ai is None:
            return self._real_solve(q)
        zr = self._real_solve(np.real(q))
        qi = np.imag(q) if np.iscomplexobj(q) else np.zeros_like(zr)
        if self.Ai is not None:
            qi = qi - self.Ai @ zr
        return zr + 1j * self._real_solve(qi)


# ---------------------------------------------------------------- quasi-Newton step
@dataclasses.dataclass
class StepResult:
    x: np.ndarray
    v: np.ndarray
    alphas: List[float]
    energies: List[float]          # f(x_k), k = 0..iters
    grad_norms: List[float]        # |g_k|, k = 0..iters
    residual: float
    status: int
    trials: int


def two_loop(g: np.ndarray, S: List[np.ndarray], Y: List[np.ndarray],
             solver: GlobalSolver) -> np.ndarray:
    """L-BFGS two-loop recursion with initial inverse Hessian H0 = A^-1 (Liu et al.
    2017); returns r = H g (the search direction is -r).  Dots run over all 3n
    components; S, Y are ordered oldest -> newest."""
    q = g.copy()
    m = len(S)
    rho = [1.0 / np.sum(Y[i] * S[i]) for i in range(m)]
    a = [0.0] * m
    for i in range(m - 1, -1, -1):
        a[i] = rho[i] * np.sum(S[i] * q)
        q = q - a[i] * Y[i]
    r = solver.solve(q)
    for i in range(m):
        b = rho[i] * np.sum(Y[i] * r)
        r = r + S[i] * (a[i] - b)
    return r


def step(rs: RestState, solver: GlobalSolver, x_n: np.ndarray, v_n: np.ndarray,
         f_ext: np.ndarray, iters: int, w_scale=None, tol: float = 0.0, contact=None, walls=None) -> StepResult:
    """One implicit time step of one cell by quasi-Newton projective dynamics.

    y = x_n + dt v_n + dt^2 M^-1 f_ext;  x^(0) = y;  history cleared.
    Repeat `iters` times: d = -two_loop(g); backtracking line search from alpha = 1
    (Armijo, or approximate Armijo g(x+ad).d <= (2 c1 - 1) g.d together with an
    energy guard f(x+ad) <= f(x) + 1e-6 |f(x)|); x <- x + alpha d; keep (s, y) when
    s.y > 1e-12 |s||y|, at most 5 pairs.  With tol > 0 (converged-residual mode, the
    iteration run towards a converged solution: Implementation and architecture
    section), stop after the first iteration whose gradient satisfies
    |g| < tol |g^(0)| (a cell with g^(0) = 0 runs all `iters`).
    v_{n+1} = (x^(k) - x_n) / dt for the last iterate k.  Works relative to the
    centroid of x_n (the objective is translation invariant), adding it back at the end.
    contact: (idx, nrm, c, delta, weight) with absolute plane offsets c (see
    detect_contacts / cell_contacts): the contact penalty joins the objective.
    walls: (lo, hi, delta, weight), box corners in absolute coordinates: the wall penalty
    of wall_energy_and_gradient joins the objective.
    With Rayleigh damping in the rest state (c_alpha, c_beta), the dissipation term of
    `objective` joins with x_n the step's start, and the solver's matrix (pd_matrix)
    carries C/dt.
    """
    dt = rs.dt
    ctr = np.real(x_n).mean(axis=0)
    xn = x_n - ctr
    y = xn + dt * v_n + dt * dt * f_ext / rs.mass[:, None]
    x = y.copy()
    if contact is not None:
        idx, nrm, c_abs, delta, weight = contact
        contact = (idx, nrm, c_abs - nrm @ ctr, delta, weight)
    if walls is not None:
        lo, hi, wdelta, wweight = walls
        walls = (np.asarray(lo, dtype=np.float64) - ctr, np.asarray(hi, dtype=np.float64) - ctr, wdelta, wweight)
    damp = (xn, damping_matrix(rs, w_scale)) if (rs.c_alpha != 0.0 or rs.c_beta != 0.0) else None
    parts, g = objective(rs, x, y, w_scale, contact, damp, walls)
    fx = parts.total
    g0n = float(np.sqrt(np.sum(np.real(g) ** 2)))
    S: List[np.ndarray] = []
    Y: List[np.ndarray] = []
    alphas, energies, gnorms = [], [fx], [g0n]
    status = STATUS_OK
    trials = 0
    for k in range(iters):
        d = -two_loop(g, S, Y, solver)
        gd = np.sum(g * d)
        if not np.real(gd) < 0.0:
            S.clear()
            Y.clear()
            d = -solver.solve(g)
            gd = np.sum(g * d)
        alpha = 1.0
        for h in range(MAX_HALVINGS + 1):
            xt = x + alpha * d
            pt, gt = objective(rs, xt, y, w_scale, contact, damp, walls)
            trials += 1
            ft = pt.total
            armijo = np.real(ft) <= np.real(fx + ARMIJO_C1 * alpha * gd)
            approx = (np.real(np.sum(gt * d)) <= np.real((2.0 * ARMIJO_C1 - 1.0) * gd)
                      and np.real(ft) <= np.real(fx) + ENERGY_GUARD_EPS * abs(np.real(fx)))
            if armijo or approx:
                break
            if h == MAX_HALVINGS:
                status |= STATUS_LINESEARCH_FAIL
                break
            alpha *= 0.5
        s = xt - x
        yy = gt - g
        if k < iters - 1:
            sy = np.real(np.sum(s * yy))
            if sy > CURVATURE_EPS * np.sqrt(np.sum(np.real(s) ** 2)) * np.sqrt(np.sum(np.real(yy) ** 2)):
                S.append(s)
                Y.append(yy)
                if len(S) > HISTORY:
                    S.pop(0)
                    Y.pop(0)
        x, g, fx = xt, gt, ft
        if pt.degenerate:
            status |= STATUS_DEGENERATE
        alphas.append(alpha)
        energies.append(float(np.real(fx)))
        gnorms.append(float(np.sqrt(np.sum(np.real(g) ** 2))))
        if tol > 0 and gnorms[-1] < tol * g0n:
            break
    residual = gnorms[-1] / g0n if g0n > 0 else 0.0
    x_new = x + ctr
    v_new = (x - xn) / dt
    if not (np.all(np.isfinite(np.real(x_new))) and np.all(np.isfinite(np.real(v_new)))):
        status |= STATUS_NONFINITE
    energies[0] = float(np.real(energies[0]))
    return StepResult(x_new, v_new, alphas, energies, gnorms, residual, status, trials)


# ---------------------------------------------------------------- batch driver
class CellType:
    """Rest state + factored global matrix of one cell type."""

    def __init__(self, verts, tris, material, dt, w_scale=None):
        """material: (w_strain, w_bend, w_area, w_vol, density[, c_alpha, c_beta[, s_min, s_max]])."""
        self.material = tuple(material)
        w_strain, w_bend, w_area, w_vol, density = material[:5]
        c_alpha, c_beta = (tuple(material[5:7]) + (0.0, 0.0))[:2]
        s_min, s_max = (tuple(material[7:9]) + (1.0, 1.0))[:2]
        self.rest = rest_state(verts, tris, w_strain, w_bend, w_area, w_vol, density, dt, c_alpha, c_beta,
                               s_min, s_max)
        self.solver = GlobalSolver(pd_matrix(self.rest, w_scale))
        self.w_scale = w_scale


def implicit_adjoint(ct: CellType, x_n: np.ndarray, v_n: np.ndarray, f_ext: np.ndarray, x_star: np.ndarray,
                     gx_next: np.ndarray, gv_next: np.ndarray):
    """Reverse-mode derivative of a loss L(x*, v*) through the converged minimiser x* of
    one step's objective (the solver run to convergence, Implementation and architecture
    section), by the implicit-function theorem instead of the unrolled iteration.

    With grad f(x*; y, w) = 0, H = grad^2 f(x*) and v* = (x* - x_n)/dt:
      H lam = dL/dx* + dL/dv* / dt,
      dL/dy = (M/dt^2) lam   (d grad f / dy = -M/dt^2),
      dL/dx_n = dL/dy - dL/dv*/dt (+ C lam / dt with Rayleigh damping),
      dL/dv_n = dt dL/dy,  dL/df = (dt^2/m) dL/dy = lam,
      dL/dw_q = -lam . d(grad f)/dw_q  for the material weights (strain, bend, area, vol).
    H and d(grad f)/dw come from complex-step differentiation of the analytic gradient
    (exact to rounding); lam from a dense solve.  With Rayleigh damping the dissipation
    term is part of f (its matrix C = c_alpha M + c_beta L(w) depends on the weights).
    Arrays [n,3]; returns gx, gv, gf, gw[4]."""
    rs = ct.rest
    dt = rs.dt
    n = rs.n
    ctr = np.real(x_n).mean(axis=0)
    xs = x_star - ctr
    y = (x_n - ctr) + dt * v_n + dt * dt * f_ext / rs.mass[:, None]
    ws0 = np.ones(4) if ct.w_scale is None else np.asarray(ct.w_scale, dtype=np.float64)
    damped = rs.c_alpha != 0.0 or rs.c_beta != 0.0
    xn = x_n - ctr

    def damp(ws):     # the step's Rayleigh dissipation term (its matrix depends on the weights)
        return (xn, damping_matrix(rs, ws)) if damped else None

    h = 1e-30
    H = np.zeros((3 * n, 3 * n))
    d0 = damp(ws0)
    for k in range(3 * n):
        e = np.zeros(3 * n, dtype=complex)
        e[k] = 1j * h
        g = objective(rs, xs + e.reshape(n, 3), y, ws0, None, d0)[1]
        H[:, k] = np.imag(g).ravel() / h
    H = 0.5 * (H + H.T)
    b = (gx_next + gv_next / dt).ravel()
    lam = np.linalg.solve(H, b).reshape(n, 3)
    dLdy = rs.mass[:, None] / dt ** 2 * lam
    gx = dLdy - gv_next / dt
    if damped:    # the dissipation term depends on x_n directly: d grad f / d x_n gains -C/dt
        gx = gx + (d0[1] @ lam) / dt
    gv = dt * dLdy
    gf = lam.copy()
    gw = np.zeros(4)
    w_mat = np.asarray(ct.material[:4], dtype=np.float64)
    for q in range(4):
        ws = ws0.astype(complex)
        ws[q] += 1j * h
        dg = np.imag(objective(rs, xs, y, ws, None, damp(ws))[1]) / h
        gw[q] = -np.sum(lam * dg) / (w_mat[q] * ws0[q])
    return gx, gv, gf, gw


def batch_step(types: List[CellType], type_of_cell, offsets, x, v, f, iters,
               cells: Optional[List[int]] = None, tol: float = 0.0,
               collisions: Optional[tuple] = None, box: Optional[tuple] = None) -> Dict[str, np.ndarray]:
    """One step for a batch in SoA [3, N_total] layout; returns new x, v (for the
    selected cells only; other columns are copied through) plus per-cell residuals,
    statuses, accepted step lengths, gradient norms and iterations done (tol: as in
    `step`).  collisions = (radius, delta, weight): contacts detected on x (for the
    selected cells' vertices) join each cell's objective; they are returned too.
    box = (lo, hi) with collisions: the box's walls act on every vertex with the same
    delta and weight."""
    xo, vo = x.copy(), v.copy()
    contacts = None
    if collisions is not None:
        radius, delta, weight = collisions
        sel = None if cells is None else [i for c in cells for i in range(int(offsets[c]), int(offsets[c + 1]))]
        contacts = detect_contacts(types, type_of_cell, offsets, x, radius, vertices=sel)
    ncells = len(type_of_cell)
    cells = range(ncells) if cells is None else cells
    res = np.zeros(ncells)
    st = np.zeros(ncells, dtype=np.int32)
    alphas, gnorms = {}, {}
    done = np.zeros(ncells, dtype=np.int32)
    for c in cells:
        s = slice(int(offsets[c]), int(offsets[c + 1]))
        ct = types[int(type_of_cell[c])]
        con = None
        if contacts is not None:
            con = (*cell_contacts(contacts, s.start, s.stop), delta, weight)
        wl = None
        if contacts is not None and box is not None:
            wl = (box[0], box[1], delta, weight)
        r = step(ct.rest, ct.solver, x[:, s].T, v[:, s].T, f[:, s].T, int(iters[c]), ct.w_scale, tol, con, wl)
        xo[:, s] = r.x.T
        vo[:, s] = r.v.T
        res[c] = r.residual
        st[c] = r.status
        alphas[c] = r.alphas
        gnorms[c] = r.grad_norms
        done[c] = len(r.alphas)
    return {"x": xo, "v": vo, "residual": res, "status": st, "alphas": alphas,
            "grad_norms": gnorms, "iters_done": done, "contacts": contacts}
