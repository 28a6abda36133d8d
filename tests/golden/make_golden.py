"""Writes the stored expected values under tests/golden/ from the oracle alone.

The paper prints no worked example (no per-vertex state or residual of any step), so the
fixtures here are the oracle's own results on seeded synthetic inputs, written by this
script, which calls only oracle/ and the seeded input generator.  They serve two checks:
the oracle still reproduces them (a change to its arithmetic shows up as a changed
fixture, regenerated only with a reason), and the CUDA path, at a rollout length the
oracle would take too long to run beside it on every GPU test, lands on them.

Fixture single_rbc_100_steps.txt: the single-RBC workload (one 642-vertex Evans-Fung RBC
at rest, axial 10 pN stretch plus 0.1 pN Gaussian noise, seed 1000, dt = 0.1 us, 5 L-BFGS
iterations per step) stepped 100 times with the same external force, in plain FP64.
Recorded: every step's residual and status, and the positions and velocities of every
8th vertex after steps 1, 10 and 100.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import npfem_oracle as O  # noqa: E402
from paper_2011_04332_b300 import inputs as I  # noqa: E402

NSTEPS = 100
RECORD_STEPS = (1, 10, 100)
VERTEX_STRIDE = 8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_rbc_100_steps.txt")


def single_rbc_rollout():
    """The oracle's rollout: per-step residuals and statuses, and the sampled states."""
    b = I.single_rbc()
    ots = [O.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt) for t in b.types]
    x, v = b.x.copy(), b.v.copy()
    residual, status, states = [], [], {}
    for s in range(1, NSTEPS + 1):
        r = O.batch_step(ots, b.type_of_cell, b.offsets, x, v, b.f, b.iters)
        x, v = r["x"], r["v"]
        residual.append(float(r["residual"][0]))
        status.append(int(r["status"][0]))
        if s in RECORD_STEPS:
            states[s] = (x[:, ::VERTEX_STRIDE].copy(), v[:, ::VERTEX_STRIDE].copy())
    return b, residual, status, states


def write(path=OUT):
    b, residual, status, states = single_rbc_rollout()
    lines = [
        "# Single-RBC rollout, plain FP64, written by tests/golden/make_golden.py (oracle only).",
        "# Method: npFEM implicit step, quasi-Newton projective dynamics with L-BFGS and line",
        "# search (Implementation and architecture section; Eq. (2) in variational form).",
        "# The paper prints no worked example; these values are the oracle's, not the paper's.",
        f"# Input: single RBC, {b.n_total} vertices, seed {b.seed}, dt {b.dt:g} us, "
        f"{int(b.iters[0])} iterations per step, {NSTEPS} steps, constant external force.",
        "# Rows:  res <step> <residual> <status>",
        f"#        x|v <step> <vertex> <c0> <c1> <c2>   (every {VERTEX_STRIDE}th vertex; SoA component order)",
    ]
    for s, (r, st) in enumerate(zip(residual, status), start=1):
        lines.append(f"res {s} {r!r} {st}")
    for s in RECORD_STEPS:
        xs, vs = states[s]
        for tag, a in (("x", xs), ("v", vs)):
            for j in range(a.shape[1]):
                lines.append(f"{tag} {s} {j * VERTEX_STRIDE} {float(a[0, j])!r} {float(a[1, j])!r} {float(a[2, j])!r}")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def read(path=OUT):
    """Parses a fixture: (residual[step], status[step], {step: (x[3, m], v[3, m])}, vertex ids)."""
    residual, status, rows = {}, {}, {}
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "res":
                residual[int(tok[1])] = float(tok[2])
                status[int(tok[1])] = int(tok[3])
            else:
                rows.setdefault((tok[0], int(tok[1])), []).append((int(tok[2]), [float(t) for t in tok[3:6]]))
    states, verts = {}, None
    for s in sorted({k[1] for k in rows}):
        ids = [r[0] for r in rows[("x", s)]]
        assert ids == [r[0] for r in rows[("v", s)]]
        verts = np.array(ids)
        states[s] = (np.array([r[1] for r in rows[("x", s)]]).T, np.array([r[1] for r in rows[("v", s)]]).T)
    return residual, status, states, verts


if __name__ == "__main__":
    write()
    print("wrote", OUT)
