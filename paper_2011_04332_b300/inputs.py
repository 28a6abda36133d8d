"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module only *generates* inputs: triangulated cell surfaces (the paper builds
its RBC/PLT meshes "through scripts using formulas", Rhino-Grasshopper section) and
per-vertex states and external forces that stand in for the immersed-boundary
coupling forces (Implementation and architecture section: the solid solver
receives external forces and returns positions and velocities).  It holds none
of the method's arithmetic: no rest geometry, masses, energies or solves.

Unit system used throughout the library: micrometre (um), microsecond (us),
picogram (pg).  Force is then pg*um/us^2 = nN, energy nN*um, and a membrane
weight (stiffness per area) nN/um.  dt = 1e-7 s = 0.1 us, 10 pN = 0.01 nN,
1.1 g/cm^3 = 1.1 pg/um^3.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

# ---------------------------------------------------------------- unit helpers
PN = 1e-3          # 1 pN in nN
UM = 1.0
US = 1.0
SECOND = 1e6       # 1 s in us
DT_DEFAULT = 1e-7 * SECOND   # 0.1 us


@dataclasses.dataclass(frozen=True)
class Material:
    """Per-cell-type weights (the per-element energy weights of the material file)."""
    w_strain: float = 1.0     # nN/um, membrane strain weight per unit rest area
    w_bend: float = 0.05      # nN*um, dihedral bending weight
    w_area: float = 10.0      # nN/um, global area weight
    w_vol: float = 10.0       # nN/um^2, global volume weight
    density: float = 1.1      # pg/um^3

    def as_tuple(self):
        return (self.w_strain, self.w_bend, self.w_area, self.w_vol, self.density)


RBC_MATERIAL = Material(1.0, 0.05, 10.0, 10.0, 1.1)
PLT_MATERIAL = Material(5.0, 0.5, 10.0, 10.0, 1.1)


@dataclasses.dataclass
class Mesh:
    """A closed, consistently (outward) oriented triangle mesh."""
    verts: np.ndarray   # float64 [n, 3], rest positions in um
    tris: np.ndarray    # int32 [T, 3]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.verts.shape[0])

    @property
    def ntris(self) -> int:
        return int(self.tris.shape[0])


# ---------------------------------------------------------------- base solids
def tetrahedron() -> Mesh:
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    v /= np.sqrt(3.0)
    t = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    return _orient_outward(Mesh(v, t, "tetrahedron"))


def icosahedron() -> Mesh:
    p = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    t = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return _orient_outward(Mesh(v, t, "icosahedron"))


def bipyramid(m: int, radius: float = 2.0, height: float = 1.0) -> Mesh:
    """Closed bipyramid over an m-gon: m equator vertices and two poles, each pole in m
    triangles (a mesh whose vertex valence exceeds any small number of colour classes)."""
    th = 2.0 * np.pi * np.arange(m) / m
    v = np.concatenate([np.stack([radius * np.cos(th), radius * np.sin(th), np.zeros(m)], axis=1),
                        [[0.0, 0.0, height], [0.0, 0.0, -height]]])
    i = np.arange(m)
    north = np.stack([i, (i + 1) % m, np.full(m, m)], axis=1)
    south = np.stack([(i + 1) % m, i, np.full(m, m + 1)], axis=1)
    return _orient_outward(Mesh(v, np.concatenate([north, south]).astype(np.int32), f"bipyramid{m}"))


def _orient_outward(m: Mesh) -> Mesh:
    """Flip every face whose normal points towards the centroid (convex base solids only)."""
    v, t = m.verts, m.tris.copy()
    c = v.mean(axis=0)
    for i in range(t.shape[0]):
        a, b, d = v[t[i, 0]], v[t[i, 1]], v[t[i, 2]]
        nrm = np.cross(b - a, d - a)
        if np.dot(nrm, (a + b + d) / 3.0 - c) < 0:
            t[i, [1, 2]] = t[i, [2, 1]]
    return Mesh(v, t, m.name)


def icosphere(subdiv: int) -> Mesh:
    """Unit icosphere: n = 10*4^s + 2 vertices, 20*4^s triangles (midpoint subdivision)."""
    m = icosahedron()
    verts = [tuple(x) for x in m.verts]
    tris = [tuple(int(i) for i in t) for t in m.tris]
    for _ in range(subdiv):
        cache = {}
        vlist = list(verts)

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            pa, pb = np.array(vlist[a]), np.array(vlist[b])
            q = (pa + pb) / 2.0
            q /= np.linalg.norm(q)
            vlist.append(tuple(q))
            cache[key] = len(vlist) - 1
            return cache[key]

        new = []
        for (a, b, c) in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        verts, tris = vlist, new
    return Mesh(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32),
                f"icosphere{subdiv}")


# ---------------------------------------------------------------- cell shapes
RBC_DIAMETER = 7.82   # um


def rbc_mesh(subdiv: int = 3, diameter: float = RBC_DIAMETER) -> Mesh:
    """Evans-Fung biconcave RBC on an icosphere.

    Shape: z = +-D*sqrt(1-rho^2)*(0.0518 + 2.0026 (r/D)^2 - 4.491 (r/D)^4), rho = 2r/D.
    A unit-sphere vertex s maps to (D/2 s_x, D/2 s_y, s_z * h(rho^2)) because
    sqrt(1-rho^2) = |s_z| on the unit sphere, so the map is smooth (no sign()).
    """
    s = icosphere(subdiv)
    R0 = diameter / 2.0
    rho2 = s.verts[:, 0] ** 2 + s.verts[:, 1] ** 2
    rd2 = rho2 / 4.0                      # (r/D)^2 with r = R0*rho
    h = diameter * (0.0518 + 2.0026 * rd2 - 4.491 * rd2 * rd2)
    v = np.stack([R0 * s.verts[:, 0], R0 * s.verts[:, 1], s.verts[:, 2] * h], axis=1)
    return Mesh(v, s.tris.copy(), f"rbc_s{subdiv}")


def platelet_mesh(subdiv: int = 2, axes=(1.8, 1.8, 0.5)) -> Mesh:
    """Oblate ellipsoid platelet (semi-axes in um) on an icosphere."""
    s = icosphere(subdiv)
    v = s.verts * np.asarray(axes, dtype=np.float64)[None, :]
    return Mesh(v, s.tris.copy(), f"plt_s{subdiv}")


# ---------------------------------------------------------------- random placement
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def stretch_forces(mesh_verts: np.ndarray, total: float = 10 * PN, frac: float = 0.05,
                   noise_sigma: float = 0.1 * PN, rng: np.random.Generator | None = None,
                   axis: int = 0) -> np.ndarray:
    """Equal and opposite uniform stretch on the `frac` extreme vertices along `axis`,
    plus Gaussian per-component noise."""
    n = mesh_verts.shape[0]
    k = max(1, int(round(frac * n)))
    order = np.argsort(mesh_verts[:, axis], kind="stable")
    f = np.zeros((n, 3))
    f[order[-k:], axis] += total / k
    f[order[:k], axis] -= total / k
    if rng is not None and noise_sigma > 0:
        f += rng.normal(0.0, noise_sigma, size=(n, 3))
    return f


def shear_noise_forces(x: np.ndarray, rng: np.random.Generator, sigma: float = 2 * PN,
                       shear_max: float = 20 * PN) -> np.ndarray:
    """Gaussian per-component forces plus a random linear shear profile
    A*((x_j - c).b / R)*a with A ~ U[0, shear_max] and a, b random orthonormal."""
    n = x.shape[0]
    f = rng.normal(0.0, sigma, size=(n, 3))
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    b = rng.standard_normal(3)
    b -= np.dot(b, a) * a
    b /= np.linalg.norm(b)
    amp = rng.uniform(0.0, shear_max)
    c = x.mean(axis=0)
    R = np.max(np.linalg.norm(x - c, axis=1))
    f += amp * (((x - c) @ b) / R)[:, None] * a[None, :]
    return f


# ---------------------------------------------------------------- batches
@dataclasses.dataclass
class CellTypeSpec:
    mesh: Mesh
    material: Material


@dataclasses.dataclass
class BatchInputs:
    """A batch of cells in SoA layout x[3][N_total] (coordinate-major), like the C ABI."""
    types: List[CellTypeSpec]
    type_of_cell: np.ndarray      # int32 [ncells]
    offsets: np.ndarray           # int64 [ncells+1] vertex offsets
    x: np.ndarray                 # float64 [3, N_total]
    v: np.ndarray                 # float64 [3, N_total]
    f: np.ndarray                 # float64 [3, N_total]
    iters: np.ndarray             # int32 [ncells]
    dt: float
    seed: int

    @property
    def ncells(self) -> int:
        return int(self.type_of_cell.shape[0])

    @property
    def n_total(self) -> int:
        return int(self.offsets[-1])

    def cell_slice(self, c: int) -> slice:
        return slice(int(self.offsets[c]), int(self.offsets[c + 1]))

    def cell_state(self, c: int):
        """(x, v, f) of one cell as [n, 3] float64 arrays."""
        s = self.cell_slice(c)
        return self.x[:, s].T.copy(), self.v[:, s].T.copy(), self.f[:, s].T.copy()

    def rbc_equivalents(self) -> float:
        """Sum over cells of (n_cell/642)*(iters_cell/5)."""
        n = np.array([self.types[t].mesh.n for t in self.type_of_cell], dtype=np.float64)
        return float(np.sum(n / 642.0 * self.iters / 5.0))


def _assemble(types, type_of_cell, xs, vs, fs, iters, dt, seed) -> BatchInputs:
    sizes = np.array([types[t].mesh.n for t in type_of_cell], dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    X = np.concatenate(xs, axis=0).T.copy() if xs else np.zeros((3, 0))
    V = np.concatenate(vs, axis=0).T.copy() if vs else np.zeros((3, 0))
    Fv = np.concatenate(fs, axis=0).T.copy() if fs else np.zeros((3, 0))
    return BatchInputs(list(types), np.asarray(type_of_cell, dtype=np.int32), offsets,
                       X, V, Fv, np.asarray(iters, dtype=np.int32), float(dt), int(seed))


def single_rbc(seed: int = 1000, subdiv: int = 3, iters: int = 5) -> BatchInputs:
    """One Evans-Fung RBC at the origin, at rest, with an axial 10 pN stretch plus
    0.1 pN noise (single-RBC workload, 642 vertices at subdivision 3)."""
    rng = np.random.default_rng(seed)
    mesh = rbc_mesh(subdiv)
    f = stretch_forces(mesh.verts, rng=rng)
    types = [CellTypeSpec(mesh, RBC_MATERIAL)]
    return _assemble(types, [0], [mesh.verts.copy()], [np.zeros_like(mesh.verts)], [f],
                     [iters], DT_DEFAULT, seed)


def placed_cells(types: Sequence[CellTypeSpec], type_of_cell: Sequence[int], seed: int,
                 iters, box: float = 200.0, dt: float = DT_DEFAULT,
                 velocity_sigma: float = 0.0) -> BatchInputs:
    """Cells with seeded random rotation + translation in a box, Gaussian + linear-shear
    forces (per cell, from SeedSequence.spawn sub-streams)."""
    ss = np.random.SeedSequence(seed)
    children = ss.spawn(len(type_of_cell))
    xs, vs, fs = [], [], []
    for c, t in enumerate(type_of_cell):
        rng = np.random.default_rng(children[c])
        mesh = types[t].mesh
        R = random_rotation(rng)
        T = rng.uniform(0.0, box, size=3)
        x = mesh.verts @ R.T + T[None, :]
        xs.append(x)
        if velocity_sigma > 0:
            vs.append(rng.normal(0.0, velocity_sigma, size=x.shape))
        else:
            vs.append(np.zeros_like(x))
        fs.append(shear_noise_forces(x, rng))
    if np.isscalar(iters):
        iters = np.full(len(type_of_cell), int(iters), dtype=np.int32)
    return _assemble(types, type_of_cell, xs, vs, fs, iters, dt, seed)


def homogeneous_rbc_batch(ncells: int = 4096, seed: int = 1001, subdiv: int = 3,
                          iters: int = 5, velocity_sigma: float = 0.0) -> BatchInputs:
    """Homogeneous batch: ncells RBCs of one 642-vertex type (4096 in the paper-scale
    workload) with random placement in a 200 um box."""
    types = [CellTypeSpec(rbc_mesh(subdiv), RBC_MATERIAL)]
    return placed_cells(types, [0] * ncells, seed, iters, velocity_sigma=velocity_sigma)


def heterogeneous_batch(n_rbc3: int = 4500, n_rbc4: int = 4500, n_plt: int = 1000,
                        seed: int = 1002, iters_range=(3, 8), shuffle: bool = True) -> BatchInputs:
    """Mixed batch: 642-vertex RBCs, 2562-vertex RBCs and 162-vertex platelets in a
    seeded random order, with a seeded per-cell iteration budget."""
    types = [CellTypeSpec(rbc_mesh(3), RBC_MATERIAL),
             CellTypeSpec(rbc_mesh(4), RBC_MATERIAL),
             CellTypeSpec(platelet_mesh(2), PLT_MATERIAL)]
    toc = np.array([0] * n_rbc3 + [1] * n_rbc4 + [2] * n_plt, dtype=np.int32)
    rng = np.random.default_rng(seed)
    if shuffle:
        rng.shuffle(toc)
    iters = rng.integers(iters_range[0], iters_range[1] + 1, size=toc.shape[0]).astype(np.int32)
    return placed_cells(types, toc, seed + 7, iters)


def stress_mix_batch(ncells: int = 20000, seed: int = 1005, iters: int = 5) -> BatchInputs:
    """Serving-shaped mix: 70 % 642-vertex RBCs, 10 % 2562-vertex RBCs and 20 % 162-vertex
    platelets in a seeded random order, `iters` iterations per cell."""
    n3 = int(round(0.7 * ncells))
    n4 = int(round(0.1 * ncells))
    return heterogeneous_batch(n3, n4, ncells - n3 - n4, seed=seed, iters_range=(iters, iters))


def redrawn_forces(b: BatchInputs, x: np.ndarray, seed: int, segment: int) -> np.ndarray:
    """A new seeded force field for the cells of `b` at positions x ([3][N_total]): the
    Gaussian + linear-shear recipe of the batch generators, drawn from the sub-streams of
    SeedSequence((seed, segment)); stands in for an updated coupling force."""
    children = np.random.SeedSequence((seed, segment)).spawn(b.ncells)
    f = np.empty_like(x)
    for c in range(b.ncells):
        s = b.cell_slice(c)
        f[:, s] = shear_noise_forces(x[:, s].T, np.random.default_rng(children[c])).T
    return f


def small_mixed_batch(seed: int = 7, iters=(2, 4, 5)) -> BatchInputs:
    """A few cells of tiny and small types for quick parity runs."""
    types = [CellTypeSpec(rbc_mesh(1), RBC_MATERIAL),
             CellTypeSpec(platelet_mesh(1), PLT_MATERIAL),
             CellTypeSpec(rbc_mesh(2), RBC_MATERIAL)]
    toc = [0, 1, 2, 0, 2, 1]
    rng = np.random.default_rng(seed)
    it = rng.integers(iters[0], iters[-1] + 1, size=len(toc)).astype(np.int32)
    return placed_cells(types, toc, seed, it, velocity_sigma=0.01)


# nominal rest volumes used only to size packing boxes (um^3): Evans-Fung RBC, platelet
RBC_NOMINAL_VOLUME = 94.1
PLT_NOMINAL_VOLUME = 6.79


def packing_batch(n_rbc: int, n_plt: int = 0, hematocrit: float = 0.35, seed: int = 1006,
                  rbc_subdiv: int = 3, plt_subdiv: int = 2, iters: int = 5) -> BatchInputs:
    """Cell-packing workload: cells at their rest shape with seeded random positions
    (uniform in a cube) and orientations, no velocity and no force.  The cube's side
    is set by the target volume fraction of the cells (nominal volumes), so randomly
    placed cells overlap; cell order: RBCs, then platelets."""
    types = [CellTypeSpec(rbc_mesh(rbc_subdiv), RBC_MATERIAL)]
    toc = [0] * n_rbc
    vol = n_rbc * RBC_NOMINAL_VOLUME
    if n_plt:
        types.append(CellTypeSpec(platelet_mesh(plt_subdiv), PLT_MATERIAL))
        toc += [1] * n_plt
        vol += n_plt * PLT_NOMINAL_VOLUME
    side = (vol / hematocrit) ** (1.0 / 3.0)
    ss = np.random.SeedSequence(seed)
    children = ss.spawn(len(toc))
    xs, vs, fs = [], [], []
    for c, t in enumerate(toc):
        rng = np.random.default_rng(children[c])
        mesh = types[t].mesh
        x = mesh.verts @ random_rotation(rng).T + rng.uniform(0.0, side, size=3)[None, :]
        xs.append(x)
        vs.append(np.zeros_like(x))
        fs.append(np.zeros_like(x))
    return _assemble(types, toc, xs, vs, fs, np.full(len(toc), iters, dtype=np.int32), DT_DEFAULT, seed)
