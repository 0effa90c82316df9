"""GPU parity of the p-multigrid transfers (Algorithm 1) for every pair of orders
1 <= p_c < p_f <= 10, through the C ABI (se_pmg_restrict, se_pmg_prolong), against the oracle.

Pairs with both N = p + 1 even run the even-odd folded kernel (J is centro-symmetric), the
others the plain one; both are covered here, in FP64 (max-norm relative error <= 1e-13, the
pMG building-block bar) and in the FP32 V-cycle's arithmetic (<= 1e-5).
"""
import numpy as np
import pytest

import oracle as o
from tests.gpu_common import Case, rel_err

pytestmark = pytest.mark.gpu

NEL = (2, 3, 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("pf", list(range(2, 11)))
def test_restrict_and_prolong_all_coarse_orders(pf, precision):
    c = Case(NEL, pf, seed=pf, bc=("D", "N", "D", "D", "N", "D"))
    se = c.se
    prec = se.SE_FP64 if precision == "fp64" else se.SE_FP32
    tol = 1e-13 if precision == "fp64" else 1e-5
    try:
        lf = c.lv
        for pc in range(1, pf):
            schedule = (pf, pc, 1) if pc > 1 else (pf, 1)
            P = se.se_pmg_setup(c.m, se.pmg_desc(schedule, se.SE_SMOOTH_JACOBI, 1, precision=prec))
            try:
                lc = o.make_level(c.V, NEL, pc, c.bc, c.amp)
                r = c.random_continuous(10 * pf + pc, lf)
                rc = c.empty(lc.gid.size)
                se.se_pmg_restrict(P, 0, c.to_gpu(r), rc)
                err_r = rel_err(c.to_np(rc, lc.gid.shape), o.restrict(lf, lc, r))
                ec = c.random_continuous(100 + 10 * pf + pc, lc)
                ef = c.empty(lf.gid.size)
                se.se_pmg_prolong(P, 0, c.to_gpu(ec), ef)
                err_p = rel_err(c.to_np(ef, lf.gid.shape), o.prolong(lf, lc, ec))
                assert err_r <= tol and err_p <= tol, (pf, pc, err_r, err_p)
            finally:
                se.se_pmg_destroy(P)
    finally:
        c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_order_transfers_with_ragged_blocks(precision):
    """p = 3 <-> 1 runs the dense small-order kernel (8 elements per block restricting, 4
    prolonging): 5 x 3 x 3 = 45 elements leave a partial last block in both directions."""
    nel = (5, 3, 3)
    c = Case(nel, 3, seed=31, bc=("D", "N", "N", "D", "D", "N"))
    se = c.se
    prec = se.SE_FP64 if precision == "fp64" else se.SE_FP32
    tol = 1e-13 if precision == "fp64" else 1e-5
    try:
        P = se.se_pmg_setup(c.m, se.pmg_desc((3, 1), se.SE_SMOOTH_JACOBI, 1, precision=prec))
        try:
            lc = o.make_level(c.V, nel, 1, c.bc, c.amp)
            r = c.random_continuous(7, c.lv)
            rc = c.empty(lc.gid.size)
            se.se_pmg_restrict(P, 0, c.to_gpu(r), rc)
            err_r = rel_err(c.to_np(rc, lc.gid.shape), o.restrict(c.lv, lc, r))
            ec = c.random_continuous(8, lc)
            ef = c.empty(c.lv.gid.size)
            se.se_pmg_prolong(P, 0, c.to_gpu(ec), ef)
            err_p = rel_err(c.to_np(ef, c.lv.gid.shape), o.prolong(c.lv, lc, ec))
            assert err_r <= tol and err_p <= tol, (err_r, err_p)
        finally:
            se.se_pmg_destroy(P)
    finally:
        c.close()
