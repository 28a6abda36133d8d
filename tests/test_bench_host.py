"""Host logic of the benchmark (no GPU): which cells its parity check samples, and the
RBC-equivalent units it counts."""
import numpy as np

import bench
from paper_2011_04332_b300 import inputs as I


def test_parity_sample_covers_every_cell_type():
    b = I.heterogeneous_batch(n_rbc3=11, n_rbc4=5, n_plt=2, seed=3)
    cells = bench.sample_cells(b)
    assert cells == sorted(set(cells))
    for t in range(3):
        idx = np.flatnonzero(b.type_of_cell == t)
        got = [c for c in cells if b.type_of_cell[c] == t]
        assert len(got) == min(3, len(idx))
        assert got[0] == idx[0] and got[-1] == idx[-1]


def test_units_weight_size_and_iterations():
    b = I.heterogeneous_batch(n_rbc3=4, n_rbc4=3, n_plt=2, seed=4)
    n = np.array([b.types[t].mesh.n for t in b.type_of_cell], float)
    assert bench.step_units(b) == np.sum(n / 642.0 * b.iters / 5.0)
    assert bench.step_units(b, tol=1e-3) == np.sum(n / 642.0)
