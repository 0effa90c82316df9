"""The library on the skewed lattice (the stand-in for the paper's Kershaw meshes, Sec. 3.1) and
with the Chebyshev bounds of the paper's sensitivity study (Table 1), against the oracle.

Checks: the operator on sheared, high-aspect-ratio elements (FP64, 1e-12); the Chebyshev-ASM and
Chebyshev-RAS smoothers with bounds away from the default, including lambda_min = 0 (Table 1's
first row, where the Chebyshev polynomial no longer damps: sigma = 1), FP64 1e-9; and whole
solves with non-default bounds: iteration counts within one of the oracle's.
"""
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, gpu, rel_err

pytestmark = pytest.mark.gpu

SMOOTHERS = {"ras": 1, "asm": 2}


@pytest.mark.parametrize("eps", [0.3, 0.05])
def test_operator_on_the_skewed_lattice(eps):
    nel = (4, 3, 4)
    c = Case(nel, 5, amp=0.0, V=wl.skewed_lattice(nel, eps))
    try:
        u = c.random_continuous(21)
        y = c.empty()
        c.se.se_ax(c.m, c.to_gpu(u), y)
        assert rel_err(c.to_np(y), o.ax(c.lv, u)) <= 1e-12
    finally:
        c.close()


@pytest.mark.parametrize("bounds", [(0.0, 1.1), (0.2, 0.95), (0.025, 1.3)])
@pytest.mark.parametrize("smoother", ["asm", "ras"])
def test_chebyshev_with_table_1_bounds(bounds, smoother):
    nel, sched = (4, 3, 3), (5, 3, 1)
    V = wl.skewed_lattice(nel, 0.3)
    c = Case(nel, 5, amp=0.0, V=V)
    se = c.se
    lo, hi = bounds
    P = se.se_pmg_setup(c.m, se.pmg_desc(sched, SMOOTHERS[smoother], 2, eig_lo=lo, eig_hi=hi))
    pmg = o.pmg_setup(V, nel, sched, smoother=smoother, order=2, eig_lo=lo, eig_hi=hi, amp=0.0)
    try:
        lam = se.se_pmg_lambda(P, 0)
        assert abs(lam - pmg.lam[0]) <= 1e-9 * pmg.lam[0]
        r = c.random_continuous(57)
        out = c.empty()
        se.se_pmg_cheby(P, 0, c.to_gpu(r), out)
        lmin, lmax = pmg.bounds[0]
        ref = o.chebyshev(r, lambda u: o.ax(pmg.levels[0], u), o.smoother_op(pmg, 0), lmin, lmax, 2)
        assert rel_err(c.to_np(out), ref) <= 1e-9
    finally:
        se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("bounds", [(0.1, 1.1), (0.2, 0.95)])
def test_solve_with_table_1_bounds_matches_the_oracle(bounds):
    nel, sched = (4, 4, 3), (5, 3, 1)
    V = wl.skewed_lattice(nel, 0.3)
    c = Case(nel, 5, amp=0.0, V=V)
    se = c.se
    lo, hi = bounds
    P = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_ASM, 2, eig_lo=lo, eig_hi=hi))
    try:
        lv, b = o.problem(V, nel, 5, amp=0.0)
        pmg = o.pmg_setup(V, nel, sched, smoother="asm", order=2, eig_lo=lo, eig_hi=hi, amp=0.0)
        xo, it_o, _ = o.solve(lv, b, pmg, tol=1e-8)
        x = c.empty().zero_()
        st = se.se_solve(c.m, P, c.to_gpu(b), x, tol=1e-8)
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        assert rel_err(c.to_np(x), xo) <= 1e-6
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_bounds_sensitivity_follows_table_1():
    """The qualitative findings of the paper's bound study (Table 1) on the skewed lattice:
    lambda_min = 0 does not converge; underestimating lambda_max costs iterations; the count is
    far less sensitive to lambda_min once it is positive.  12^3 elements, p = 7, (7,3,1)
    Cheby-ASM(2), FP32 V-cycle, GMRES(20) to 1e-8."""
    import bench
    torch, se = gpu()
    m, info, b = bench.skewed_problem(se, torch, (12, 12, 12), 7, 0.3)
    its = {}
    try:
        for lo, hi in [(0.0, 1.1), (0.1, 0.9), (0.1, 1.1), (0.2, 1.1), (0.05, 1.2), (0.025, 0.95),
                       (0.025, 1.1)]:
            d = se.pmg_desc((7, 3, 1), se.SE_SMOOTH_ASM, 2, eig_lo=lo, eig_hi=hi, precision=se.SE_FP32)
            ok, st = bench.study_solve(se, torch, m, b, d, se.SE_FGMRES, 300)
            its[(lo, hi)] = st.iterations if ok else None
    finally:
        se.se_mesh_destroy(m)
    assert its[(0.0, 1.1)] is None, its
    base = its[(0.1, 1.1)]
    assert base is not None and base < 100, its
    assert its[(0.1, 0.9)] is None or its[(0.1, 0.9)] > base, its
    assert its[(0.025, 0.95)] is None or its[(0.025, 0.95)] > its[(0.025, 1.1)], its
    for k in [(0.2, 1.1), (0.05, 1.2)]:
        assert its[k] is not None and abs(its[k] - base) <= 0.35 * base, its
