"""Double-float (df64) arithmetic for the two arithmetic-bound kernels, against the FP64 oracle.

GB300 runs FP32 FMAs at 64 times its FP64 rate, so the sum-factorised operator and the FDM
solves also run in df64 (pairs of FP32 values, about 48 significant bits) on FP64 vectors.  The
bar is the FP64 one: operator relative error <= 1e-12 (every p = 1..10, ragged meshes, all flag
combinations, Neumann and Dirichlet faces); FDM smoother <= 1e-10 and Chebyshev <= 1e-9 as for
FP64; whole solves with the SE_DF64 preconditioner and the df64 outer operator: iteration counts
within +-1 of the oracle, true residual <= 1.5e-8, and the device-driven graph equal to the host
loop bit for bit.  Odd orders use the even-odd folded operator, even orders the plain sum
factorisation kernel in df64.
"""
import math

import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, rel_err

pytestmark = pytest.mark.gpu

ORDERS = [((1, 1, 1), 1), ((3, 2, 2), 3), ((2, 3, 3), 5), ((3, 1, 2), 7), ((2, 2, 1), 9),
          ((5, 4, 3), 3), ((4, 3, 4), 7), ((2, 2, 2), 2), ((3, 2, 2), 4), ((2, 3, 1), 6),
          ((2, 1, 2), 8), ((1, 2, 1), 10)]


@pytest.mark.parametrize("nel,p", ORDERS)
@pytest.mark.parametrize("bc", [("D",) * 6, ("N", "D", "N", "N", "D", "N")])
def test_df64_operator(nel, p, bc):
    c = Case(nel, p, seed=50 + p, bc=bc)
    se = c.se
    try:
        u = c.random_continuous(7, masked=False)
        ug, y = c.to_gpu(u), c.empty()
        DF = se.SE_AX_DF64
        se.se_ax(c.m, ug, y, se.SE_AX_ASSEMBLE | se.SE_AX_MASK | DF)
        assert rel_err(c.to_np(y), o.ax(c.lv, u)) <= 1e-12
        se.se_ax(c.m, ug, y, DF)
        assert rel_err(c.to_np(y), o.ax_local(c.lv, u)) <= 1e-12
        se.se_ax(c.m, ug, y, se.SE_AX_ASSEMBLE | DF)
        assert rel_err(c.to_np(y), o.ax(c.lv, u, mask=False)) <= 1e-12
        # the df64 result is not the FP64 one bit for bit, but agrees to about 1e-14
        y64 = c.empty()
        se.se_ax(c.m, ug, y64, se.SE_AX_ASSEMBLE)
        assert rel_err(c.to_np(y), c.to_np(y64)) <= 1e-13
    finally:
        c.close()


SMOOTHERS = {"ras": 1, "asm": 2, "jacobi": 0}


@pytest.mark.parametrize("nel,p,schedule", [((3, 2, 2), 5, (5, 3, 1)), ((2, 3, 2), 7, (7, 3, 1)),
                                            ((2, 2, 2), 9, (9, 5, 1)), ((2, 2, 3), 6, (6, 3, 1)),
                                            ((2, 2, 2), 10, (10, 4, 2, 1))])
@pytest.mark.parametrize("smoother", ["ras", "asm"])
def test_df64_smoother_and_chebyshev(nel, p, schedule, smoother):
    c = Case(nel, p, seed=3)
    se = c.se
    P = se.se_pmg_setup(c.m, se.pmg_desc(schedule, SMOOTHERS[smoother], 2, precision=se.SE_DF64))
    pmg = o.pmg_setup(c.V, nel, schedule, smoother=smoother, order=2, amp=c.amp)
    try:
        for l in range(len(schedule) - 1):
            lv = pmg.levels[l]
            lam = se.se_pmg_lambda(P, l)
            assert abs(lam - pmg.lam[l]) <= 1e-9 * pmg.lam[l]
            r = c.random_continuous(60 + l, lv)
            out = c.empty(lv.gid.size)
            se.se_pmg_smooth(P, l, c.to_gpu(r), out)
            assert rel_err(c.to_np(out, lv.gid.shape), o.smoother_op(pmg, l)(r)) <= 1e-10
            se.se_pmg_level_ax(P, l, c.to_gpu(r), out)
            assert rel_err(c.to_np(out, lv.gid.shape), o.ax(lv, r)) <= 1e-12
        r = c.random_continuous(33)
        out = c.empty()
        se.se_pmg_cheby(P, 0, c.to_gpu(r), out)
        lmin, lmax = pmg.bounds[0]
        ref = o.chebyshev(r, lambda u: o.ax(pmg.levels[0], u), o.smoother_op(pmg, 0), lmin, lmax, 2)
        assert rel_err(c.to_np(out), ref) <= 1e-9
    finally:
        se.se_pmg_destroy(P)
        c.close()


def gpu_rhs(c):
    xyz = c.empty(3 * c.info.L)
    c.se.se_mesh_nodes(c.m, xyz)
    X = xyz.cpu().numpy().reshape(3, -1)
    b = c.empty()
    c.se.se_mesh_rhs(c.m, c.to_gpu(wl.f_rhs(X[0], X[1], X[2])), b)
    return b


@pytest.mark.parametrize("smoother,method", [("ras", "fpcg"), ("jacobi", "fpcg"), ("asm", "fgmres")])
def test_df64_solve_parity(smoother, method):
    c = Case((4, 4, 3), 7, pert=0.05, seed=2)
    se = c.se
    sched = (7, 5, 3, 1) if smoother == "jacobi" else (7, 3, 1)
    P = se.se_pmg_setup(c.m, se.pmg_desc(sched, SMOOTHERS[smoother], 2, precision=se.SE_DF64))
    try:
        b = gpu_rhs(c)
        lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
        pmg = o.pmg_setup(c.V, c.nel, sched, smoother=smoother, order=2, amp=c.amp)
        xo, it_o, _ = o.solve(lvo, bo, pmg, method=method, tol=1e-8)
        meth = se.SE_FPCG if method == "fpcg" else se.SE_FGMRES
        x = c.empty().zero_()
        st = se.se_solve(c.m, P, b, x, method=meth, tol=1e-8, operator_df64=1)
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        r = bo - o.ax(lvo, c.to_np(x))
        assert math.sqrt(o.dot(lvo, r, r) / o.dot(lvo, bo, bo)) <= 1.5e-8
        assert rel_err(c.to_np(x), xo) <= 1e-6
        if method == "fpcg":
            xg = c.empty().zero_()
            sg = se.se_solve(c.m, P, b, xg, tol=1e-8, operator_df64=1, graph_capture=1)
            assert sg.iterations == st.iterations and c.torch.equal(xg, x)
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_df64_operator_in_a_batch_matches_each_solve_alone():
    """Batched solves with the df64 outer operator (problems grouped by preconditioner
    configuration, the group's outer operator in df64): each problem meets the tolerance and
    agrees with its own df64-operator graph solve and with the FP64-operator solve to within
    rounding (iterations within one)."""
    from tests.gpu_common import gpu
    torch, se = gpu()
    probs = []
    try:
        for nel, p, sched, seed in [((3, 3, 2), 5, (5, 3, 1), 1), ((2, 3, 3), 7, (7, 3, 1), 2),
                                    ((3, 2, 3), 7, (7, 3, 1), 3)]:
            c = Case(nel, p, seed=seed)
            P = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32))
            probs.append((c, P, gpu_rhs(c), c.empty().zero_()))
        B = se.se_batch_create([(c.m, P, b, x) for c, P, b, x in probs], tol=1e-8, maxit=200,
                               operator_df64=1)
        try:
            assert se.se_batch_info(B) == (2, 3)
            se.se_batch_run(B)
            stats = se.se_batch_stats(B, len(probs))
        finally:
            se.se_batch_destroy(B)
        for (c, P, b, x), sb in zip(probs, stats):
            assert sb.rel_residual <= 1e-8
            xa = c.empty().zero_()
            st = se.se_solve(c.m, P, b, xa, tol=1e-8, graph_capture=1, operator_df64=1)
            assert abs(sb.iterations - st.iterations) <= 1
            assert rel_err(c.to_np(x), c.to_np(xa)) <= 1e-6
            x64 = c.empty().zero_()
            st64 = se.se_solve(c.m, P, b, x64, tol=1e-8)
            assert abs(st.iterations - st64.iterations) <= 1
            assert rel_err(c.to_np(x), c.to_np(x64)) <= 1e-6
    finally:
        for c, P, b, x in probs:
            se.se_pmg_destroy(P)
            c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_arnoldi_in_df64_gives_the_same_bounds(precision):
    """arnoldi_df64: the eigenvalue estimate of an FP64 or FP32 preconditioner with df64 operator
    and FDM arithmetic agrees with the FP64 one and the oracle's to 1e-9 (the df64 copies are
    set-up transients); the V-cycle itself is unchanged: bit for bit the same as without."""
    c = Case((3, 2, 3), 7, seed=4)
    se = c.se
    sched = (7, 3, 1)
    P0 = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 2, precision=precision))
    P1 = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 2, precision=precision,
                                          arnoldi_df64=1))
    pmg = o.pmg_setup(c.V, c.nel, sched, smoother="ras", order=2, amp=c.amp)
    try:
        for l in range(len(sched) - 1):
            l0, l1 = se.se_pmg_lambda(P0, l), se.se_pmg_lambda(P1, l)
            assert abs(l1 - l0) <= 1e-11 * l0 and abs(l1 - pmg.lam[l]) <= 1e-9 * pmg.lam[l]
        r = c.to_gpu(c.random_continuous(12))
        z0, z1 = c.empty(), c.empty()
        se.se_pmg_smooth(P0, 0, r, z0)
        se.se_pmg_smooth(P1, 0, r, z1)
        assert c.torch.equal(z0, z1)
    finally:
        se.se_pmg_destroy(P0)
        se.se_pmg_destroy(P1)
        c.close()


@pytest.mark.parametrize("scale", [2.0 ** -70, 2.0 ** -30, 1.0, 2.0 ** 40])
def test_df64_operator_across_the_supported_range(scale):
    """Inputs anywhere in the df64 range (|u| in [2^-103, 2^128), operator output within it too)
    keep the FP64 bar; exact zeros (the Dirichlet copies of a masked vector) stay exact."""
    c = Case((3, 2, 2), 5, seed=21)
    se = c.se
    try:
        u = c.random_continuous(3) * scale
        y = c.empty()
        se.se_ax(c.m, c.to_gpu(u), y, se.SE_AX_ASSEMBLE | se.SE_AX_MASK | se.SE_AX_DF64)
        ref = o.ax(c.lv, u)
        assert rel_err(c.to_np(y), ref) <= 1e-12
        assert (c.to_np(y)[c.lv.mask == 0] == 0).all()
    finally:
        c.close()
