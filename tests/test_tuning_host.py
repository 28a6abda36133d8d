"""Host logic of the launch-shape autotuner: every candidate it would time fits the SM's
shared memory and warp budgets stated by the generators, for the mesh sizes of the
workloads (42- and 162-vertex test meshes, 642-vertex RBC, 2562-vertex RBC)."""
import pytest

from paper_2011_04332_b300 import tuning as T

SMEM_SM, SMEM_CTA = 228 * 1024, 227 * 1024
SIZES = (42, 162, 642, 2562)


@pytest.mark.parametrize("n", SIZES)
def test_split_solve_candidates_fit(n):
    cands = T.split_solve_candidates(n)
    assert cands and len(cands) == len(set(cands))
    for wpb, bps, place, per_coord, cells in cands:
        warps = wpb * bps
        assert warps >= 4 and bps <= 16, (wpb, bps)
        if place == 2:                         # one interleaved vector per cell of the CTA
            zb = 24 * (n + 1) * cells
            assert cells in (1, 2) and per_coord == 0 and wpb in ((2, 4, 6, 8) if cells == 1 else (2, 4))
            assert zb <= SMEM_CTA and bps * (zb + 1024) <= SMEM_SM
            assert bps <= (T.CTA_MAX_CTAS if cells == 1 else T.CTA2_MAX_CTAS)[wpb]
        elif place == 1:                       # per-warp vectors in shared memory
            zb = (8 if per_coord else 24) * (n + 1)
            cta = wpb * cells * zb
            assert cta <= SMEM_CTA and bps * (cta + 1024) <= SMEM_SM
            assert warps <= T.SOLVE_MAX_WARPS[cells] and warps * cells >= 8
        else:                                  # vectors in the workspace
            assert place == 0 and per_coord == 0 and cells != 3
            assert warps in (8, 16, 24, 32) and warps <= T.SOLVE_MAX_WARPS[cells]


def test_cta_cooperative_solve_offered_for_every_workload_size():
    for n in SIZES:
        assert any(c[2] == 2 for c in T.split_solve_candidates(n)), n


@pytest.mark.parametrize("n", SIZES)
def test_fused_mode_candidates_fit(n):
    for wpb, bps, in_smem, per_coord in T.candidate_shapes(n):
        assert wpb * bps >= 3
        if in_smem:
            zb = (8 if per_coord else 24) * (n + 1)
            assert wpb * zb <= SMEM_CTA and bps * wpb * zb <= SMEM_SM


def test_iteration_kernel_candidates():
    cands = T.split_iter_candidates()
    assert (2, 16) in cands                    # the FP32 form's 32 warps per SM
    for wpb, bps in cands:
        assert wpb in (2, 4) and 8 <= wpb * bps <= 32 and (wpb * bps) % 4 == 0
