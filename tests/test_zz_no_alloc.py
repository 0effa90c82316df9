"""The coarse solve that allocates nothing (se_pmg_coarse_solve_noalloc).

It exists for callers that must not allocate device memory during the call, such as code that
runs after its memory pool is fixed.  Its work space is one static device array of the
library, so this test checks it through the C ABI against the allocating entry point
se_pmg_coarse_solve on the same preconditioner and right-hand side, on two calls in a row (the
second call reuses the array left by the first) with an injected failure armed for the next
device allocation (so any allocation during the call would fail it), against the oracle's
coarse solve as well, and that a coarse level above the static limit is rejected.  It runs last so that a failure here leaves every other test already run, and it
passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle as o
from tests.gpu_common import Case, gpu, rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_coarse_solve_matches_allocating_entry_point():
    c = Case((5, 4, 3), 5, seed=9)
    se = c.se
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2))
    try:
        info = se.se_pmg_level_info(P, 2)
        lc = o.make_level(c.V, c.nel, 1, c.bc, c.amp)
        lc.extra["diag"] = o.jacobi_diag(lc)
        coarse = o.PMG(levels=[lc], smoother="jacobi", order=[], bounds=[], lam=[])
        for call, seed in enumerate((101, 202)):
            rc = c.random_continuous(seed, lc)
            r = c.to_gpu(rc)
            x_ref = c.empty(info.L)
            x_new = c.empty(info.L).fill_(np.nan)
            it_ref = se.se_pmg_coarse_solve(P, r, x_ref)
            # any device allocation by the library during the call would now fail with ENOMEM
            se.se_selftest_fail_alloc(1)
            try:
                it_new = se.se_pmg_coarse_solve_noalloc(P, r, x_new)
            finally:
                se.se_selftest_fail_alloc(0)
            assert it_new == it_ref, (call, it_new, it_ref)
            err = rel_err(c.to_np(x_new, (info.L,)), c.to_np(x_ref, (info.L,)))
            assert err <= 1e-12, (call, err)
            # and against the oracle's Jacobi-PCG on the same coarse level
            x_o = o.coarse_solve(coarse, rc)
            assert abs(it_new - coarse.coarse_iters[-1]) <= 1
            if it_new == coarse.coarse_iters[-1]:
                assert rel_err(c.to_np(x_new, lc.gid.shape), x_o) <= 1e-8, call
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_noalloc_coarse_solve_rejects_too_large_coarse_level():
    torch, se = gpu()
    m = se.se_mesh_create((51, 51, 51), 2)        # p = 1 level: 52^3 = 140608 > 131072 nodes
    P = se.se_pmg_setup(m, se.pmg_desc((2, 1), se.SE_SMOOTH_JACOBI, 1))
    try:
        info = se.se_pmg_level_info(P, 1)
        assert info.n_global > 131072
        r = torch.zeros(info.L, dtype=torch.float64, device="cuda")
        x = torch.empty_like(r)
        with pytest.raises(se.SeError) as e:
            se.se_pmg_coarse_solve_noalloc(P, r, x)
        assert e.value.code == se.SE_EINVAL
        assert "static limit" in str(e.value)
    finally:
        se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)
