"""Launch-tile autotuner: the measured choice is a valid tile, and results do not depend on the
tile (every element is computed by one block, so outputs are bitwise identical)."""
import pytest

from tests.gpu_common import Case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [3, 7])
@pytest.mark.parametrize("prec", [0, 1])
def test_tune_valid_and_results_tile_independent(p, prec):
    c = Case((3, 3, 2), p, seed=2)
    se, torch = c.se, c.torch
    try:
        P = se.se_pmg_setup(c.m, se.pmg_desc((p, 1), se.SE_SMOOTH_RAS, 1, precision=prec))
        u = c.to_gpu(c.random_continuous(3))
        y0, y1, z0, z1 = c.empty(), c.empty(), c.empty(), c.empty()
        flags = se.SE_AX_ASSEMBLE | se.SE_AX_MASK | (se.SE_AX_FP32 if prec else 0)
        se.se_ax(c.m, u, y0, flags)
        se.se_pmg_smooth(P, 0, u, z0)
        cfg = se.se_tune(p, prec)
        N, PB = p + 1, p + 3
        assert 1 <= cfg.ax_elems_per_block and cfg.ax_elems_per_block * N * N <= 512
        # FP64 FDM: one thread per line of every element in the block; FP32: one warp per element
        fdm_threads = cfg.fdm_elems_per_block * (32 if prec else PB * PB)
        assert 1 <= cfg.fdm_elems_per_block <= 16 and fdm_threads <= (256 if prec else 512)
        assert cfg.ax_ms > 0 and cfg.fdm_ms > 0
        got = se.se_tune_get(p, prec)
        assert (got.ax_elems_per_block, got.fdm_elems_per_block) == (cfg.ax_elems_per_block, cfg.fdm_elems_per_block)
        for ax_ne, fdm_ne in [(1, 1), (2, 3), (3, 8 if prec else 2)]:
            se.se_tune_set(p, prec, ax_ne, fdm_ne)
            se.se_ax(c.m, u, y1, flags)
            se.se_pmg_smooth(P, 0, u, z1)
            assert torch.equal(y0, y1)
            assert torch.equal(z0, z1)
        se.se_tune_set(p, prec, 0, 0)
        se.se_pmg_destroy(P)
    finally:
        c.close()
