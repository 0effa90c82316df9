"""GPU parity of the p-multigrid building blocks (Sec. 2.2, Algorithms 1-2, eqs 4-9).

Tolerances (relative, max-norm): gather and transfers 1e-13; smoothers, FDM, Chebyshev 1e-10
(the local eigen-decompositions are computed by different algorithms: cyclic Jacobi rotations
on the GPU, LAPACK eigh in the oracle; the FDM result is invariant to them up to rounding
times the local condition number); lambda-tilde 1e-9; V-cycle 1e-8 when both coarse solves
take the same number of iterations.  FP32 preconditioner against the FP64 oracle: 1e-4.
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, gpu, rel_err

pytestmark = pytest.mark.gpu

SMOOTHERS = {"ras": 1, "asm": 2, "jacobi": 0}


def build(nel, p, schedule, smoother, order=2, precision=0, seed=3, bc=("D",) * 6):
    c = Case(nel, p, seed=seed, bc=bc)
    se = c.se
    P = se.se_pmg_setup(c.m, se.pmg_desc(schedule, SMOOTHERS[smoother], order, precision=precision))
    pmg = o.pmg_setup(c.V, nel, schedule, smoother=smoother, order=order, bc=bc, amp=c.amp)
    return c, P, pmg


CASES = [((3, 2, 2), 5, (5, 3, 1)), ((2, 3, 2), 7, (7, 3, 1)), ((2, 2, 2), 9, (9, 5, 1)),
         ((4, 3, 2), 3, (3, 1))]


@pytest.mark.parametrize("nel,p,schedule", CASES)
@pytest.mark.parametrize("smoother", ["ras", "jacobi", "asm"])
def test_pmg_building_blocks(nel, p, schedule, smoother):
    c, P, pmg = build(nel, p, schedule, smoother)
    se, torch = c.se, c.torch
    try:
        for l in range(len(schedule) - 1):
            lv = pmg.levels[l]
            info = se.se_pmg_level_info(P, l)
            assert info.L == lv.gid.size
            lam = se.se_pmg_lambda(P, l)
            assert abs(lam - pmg.lam[l]) <= 1e-9 * pmg.lam[l], (lam, pmg.lam[l])
            r = c.random_continuous(40 + l, lv)
            rg = c.to_gpu(r)
            out = c.empty(info.L)
            se.se_pmg_level_ax(P, l, rg, out)
            assert rel_err(c.to_np(out, lv.gid.shape), o.ax(lv, r)) <= 1e-12
            se.se_pmg_smooth(P, l, rg, out)
            ref = o.smoother_op(pmg, l)(r)
            assert rel_err(c.to_np(out, lv.gid.shape), ref) <= 1e-10
            se.se_pmg_cheby(P, l, rg, out)
            lmin, lmax = pmg.bounds[l]
            refc = o.chebyshev(r, lambda u: o.ax(lv, u), o.smoother_op(pmg, l), lmin, lmax, 2)
            assert rel_err(c.to_np(out, lv.gid.shape), refc) <= 1e-9
            # transfers to/from the next level
            lc = pmg.levels[l + 1]
            rc = c.empty(lc.gid.size)
            se.se_pmg_restrict(P, l, rg, rc)
            assert rel_err(c.to_np(rc, lc.gid.shape), o.restrict(lv, lc, r)) <= 1e-13
            ec = c.random_continuous(50 + l, lc)
            se.se_pmg_prolong(P, l, c.to_gpu(ec), out)
            assert rel_err(c.to_np(out, lv.gid.shape), o.prolong(lv, lc, ec)) <= 1e-13
            if smoother != "jacobi":
                pb = lv.p + 3
                rbar = c.empty(lv.E * pb ** 3)
                se.se_pmg_gather_ext(P, l, rg, rbar)
                ref_bar = o.extended_gather(lv, r)
                assert rel_err(c.to_np(rbar, ref_bar.shape), ref_bar) <= 1e-15
                xb = wl.random_lvector(ref_bar.shape, 60 + l)
                zb = c.empty(lv.E * pb ** 3)
                se.se_pmg_fdm(P, l, c.to_gpu(xb), zb)
                S, Lm = lv.extra["fdm"]
                assert rel_err(c.to_np(zb, ref_bar.shape), o.fdm_apply(S, Lm, xb)) <= 1e-10
        # coarse solve and the whole V-cycle
        lcs = pmg.levels[-1]
        rc = c.random_continuous(70, lcs)
        xc = c.empty(lcs.gid.size)
        it = se.se_pmg_coarse_solve(P, c.to_gpu(rc), xc)
        pmg.coarse_iters.clear()
        xref = o.coarse_solve(pmg, rc)
        it_ref = pmg.coarse_iters[-1]
        assert abs(it - it_ref) <= 1
        if it == it_ref:
            assert rel_err(c.to_np(xc, lcs.gid.shape), xref) <= 1e-8
        lv0 = pmg.levels[0]
        r0 = c.random_continuous(80, lv0)
        z = c.empty()
        se.se_pmg_apply(P, c.to_gpu(r0), z)
        pmg.coarse_iters.clear()
        zref = o.vcycle(pmg, r0)
        assert rel_err(c.to_np(z), zref) <= 1e-6
        torch.cuda.synchronize()
    finally:
        se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("smoother", ["ras", "jacobi", "asm"])
def test_fp32_vcycle_against_fp64_oracle(smoother):
    c, P, pmg = build((3, 2, 2), 7, (7, 3, 1), smoother, precision=1)
    try:
        r0 = c.random_continuous(90)
        z = c.empty()
        c.se.se_pmg_apply(P, c.to_gpu(r0), z)
        zref = o.vcycle(pmg, r0)
        assert rel_err(c.to_np(z), zref) <= 1e-4
        assert abs(c.se.se_pmg_lambda(P, 0) - pmg.lam[0]) <= 1e-9 * pmg.lam[0]
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("smoother", ["ras", "asm"])
def test_additive_vcycle_against_oracle(smoother, precision):
    """The additive V-cycle (Sec. 2.2.2: Schwarz smoothers without Chebyshev acceleration,
    x = S b + P V(P^T b), no post-smoothing) through se_pmg_apply, against the oracle's:
    FP64 and df64 within the V-cycle bar 1e-6 (the coarse Jacobi-PCG iterations may differ by
    one), the FP32 V-cycle within 1e-4."""
    nel, p, sched = (3, 2, 2), 7, (7, 3, 1)
    c = Case(nel, p, seed=3)
    se = c.se
    P = se.se_pmg_setup(c.m, se.pmg_desc(sched, SMOOTHERS[smoother], 0, precision=precision,
                                          cycle=se.SE_CYCLE_ADDITIVE))
    pmg = o.pmg_setup(c.V, nel, sched, smoother=smoother, order=0, amp=c.amp, cycle="additive")
    try:
        r = c.random_continuous(77)
        z = c.empty()
        se.se_pmg_apply(P, c.to_gpu(r), z)
        assert rel_err(c.to_np(z), o.vcycle(pmg, r)) <= (1e-4 if precision == 1 else 1e-6)
    finally:
        se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("method", ["fpcg", "fgmres"])
def test_additive_vcycle_solve(method):
    """FPCG / FGMRES(20) preconditioned by the additive RAS cycle on the 4^3 p = 7 box: the
    oracle's iteration count within one, the tolerance met by the true residual."""
    c = Case((4, 4, 4), 7, pert=0.0)
    se = c.se
    sched = (7, 3, 1)
    P = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 0, cycle=se.SE_CYCLE_ADDITIVE))
    try:
        xyz = c.empty(3 * c.info.L)
        se.se_mesh_nodes(c.m, xyz)
        X = xyz.cpu().numpy().reshape(3, -1)
        b = c.empty()
        se.se_mesh_rhs(c.m, c.to_gpu(wl.f_rhs(X[0], X[1], X[2])), b)
        x = c.empty().zero_()
        meth = se.SE_FPCG if method == "fpcg" else se.SE_FGMRES
        st = se.se_solve(c.m, P, b, x, method=meth, tol=1e-8, maxit=500, restart=20)
        lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
        pmg = o.pmg_setup(c.V, c.nel, sched, smoother="ras", order=0, amp=c.amp, cycle="additive")
        xo, it_o, _ = o.solve(lvo, bo, pmg, method=method, tol=1e-8, maxit=500)
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        r = bo - o.ax(lvo, c.to_np(x))
        assert math.sqrt(o.dot(lvo, r, r) / o.dot(lvo, bo, bo)) <= 1.5e-8
        assert rel_err(c.to_np(x), xo) <= 1e-5
    finally:
        se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("smoother", ["ras", "jacobi"])
def test_chebyshev_orders(order, smoother, precision):
    """Algorithm 2 at every Chebyshev order the tests use (0 = the plain smoother step r/theta);
    the first step applies A and S to r and scales by 1/theta, the last one folds in the final
    x += d.  FP64 1e-9 (as the other smoother checks); FP32 1e-4."""
    c, P, pmg = build((3, 2, 2), 5, (5, 3, 1), smoother, order=order, precision=precision)
    try:
        lv = pmg.levels[0]
        r = c.random_continuous(33)
        out = c.empty()
        c.se.se_pmg_cheby(P, 0, c.to_gpu(r), out)
        lmin, lmax = pmg.bounds[0]
        ref = o.chebyshev(r, lambda u: o.ax(lv, u), o.smoother_op(pmg, 0), lmin, lmax, order)
        assert rel_err(c.to_np(out, lv.gid.shape), ref) <= (1e-4 if precision else 1e-9)
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("p", range(2, 11))
@pytest.mark.parametrize("smoother", ["ras", "asm"])
def test_fp32_schwarz_smoother_all_orders(p, smoother):
    """FP32 Schwarz smoother (one warp per element: gather, six contractions, D^-1, RAS
    weights or ASM combine, QQ^T) at every order the library takes, on 12 elements (a block of
    8 and a partial one), against the FP64 oracle at the FP32 preconditioner tolerance 1e-4."""
    c, P, pmg = build((3, 2, 2), p, (p, 1), smoother, precision=1)
    try:
        r = c.random_continuous(95 + p)
        out = c.empty()
        c.se.se_pmg_smooth(P, 0, c.to_gpu(r), out)
        ref = o.smoother_op(pmg, 0)(r)
        assert rel_err(c.to_np(out), ref) <= 1e-4
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("p", range(2, 11))
@pytest.mark.parametrize("smoother", ["ras", "asm", "jacobi"])
def test_fp64_smoother_all_orders(p, smoother):
    """FP64 smoothers (Schwarz: window gather, FDM, RAS weights or ASM combine, QQ^T; Jacobi)
    and their Arnoldi bound at every order the library takes, odd and even p, on 12 elements
    with mixed boundary conditions, against the oracle at the FP64 smoother bar 1e-10."""
    bc = ("D", "N", "D", "D", "N", "D")
    c, P, pmg = build((3, 2, 2), p, (p, 1), smoother, bc=bc)
    try:
        r = c.random_continuous(195 + p)
        out = c.empty()
        c.se.se_pmg_smooth(P, 0, c.to_gpu(r), out)
        assert rel_err(c.to_np(out), o.smoother_op(pmg, 0)(r)) <= 1e-10
        lam = c.se.se_pmg_lambda(P, 0)
        assert abs(lam - pmg.lam[0]) <= 1e-9 * pmg.lam[0]
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


def test_fp32_ras_mixed_boundaries():
    bc = ("D", "N", "N", "D", "N", "D")
    c, P, pmg = build((2, 3, 2), 7, (7, 3, 1), "ras", precision=1, bc=bc)
    try:
        r = c.random_continuous(97)
        out = c.empty()
        c.se.se_pmg_smooth(P, 0, c.to_gpu(r), out)
        assert rel_err(c.to_np(out), o.smoother_op(pmg, 0)(r)) <= 1e-4
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


def test_two_preconditioners_on_one_mesh():
    c = Case((2, 2, 2), 5)
    se = c.se
    try:
        P1 = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2))
        P2 = se.se_pmg_setup(c.m, se.pmg_desc((5, 1), se.SE_SMOOTH_JACOBI, 3))
        r = c.to_gpu(c.random_continuous(1))
        z1, z2, z3 = c.empty(), c.empty(), c.empty()
        se.se_pmg_apply(P1, r, z1)
        se.se_pmg_apply(P2, r, z2)
        se.se_pmg_destroy(P2)
        se.se_pmg_apply(P1, r, z3)
        assert c.torch.equal(z1, z3)
        se.se_pmg_destroy(P1)
    finally:
        c.close()


def test_coarse_stats_count_solves_and_iterations():
    """se_pmg_coarse_stats counts every coarse solve and its Jacobi-PCG iterations, on the device,
    including those inside V-cycles (one per V-cycle), and resets on request."""
    c = Case((3, 3, 2), 5, seed=3)
    se, torch = c.se, c.torch
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2))
    try:
        se.se_pmg_coarse_stats(P, reset=True)
        lc = o.make_level(c.V, c.nel, 1, c.bc, c.amp)
        info = se.se_pmg_level_info(P, 2)
        it1 = se.se_pmg_coarse_solve(P, c.to_gpu(c.random_continuous(5, lc)), c.empty(info.L))
        it2 = se.se_pmg_coarse_solve(P, c.to_gpu(c.random_continuous(6, lc)), c.empty(info.L))
        assert se.se_pmg_coarse_stats(P) == (2, it1 + it2)
        z = c.empty()
        se.se_pmg_apply(P, c.to_gpu(c.random_continuous(7)), z)
        n, its = se.se_pmg_coarse_stats(P, reset=True)
        assert n == 3 and its > it1 + it2
        assert se.se_pmg_coarse_stats(P) == (0, 0)
    finally:
        se.se_pmg_destroy(P)
        c.close()


@pytest.mark.gpu
@pytest.mark.parametrize("nel", [(37, 37, 37), (43, 43, 43)])
def test_large_coarse_solves_against_the_oracle(nel):
    """The coarse Jacobi-PCG at sizes where the solver's two kernels take over: 38^3 = 54,872
    nodes run one node per thread (row of Ahat in shared memory, per-block neighbour flags, a
    grid of two blocks per SM); 44^3 = 85,184 nodes exceed the co-resident threads and run the
    grid-strided kernel.  Iterations within one of the oracle's, solution to 1e-8."""
    torch, se = gpu()
    V = wl.vertex_lattice(nel, 0.05, 2)
    m = se.se_mesh_create(nel, 2, vertex_xyz=V, deform_amp=wl.DEFORM_AMP)
    P = se.se_pmg_setup(m, se.pmg_desc((2, 1), se.SE_SMOOTH_JACOBI, 1))
    try:
        lc = o.make_level(V, nel, 1, ("D",) * 6, wl.DEFORM_AMP)
        lc.extra["diag"] = o.jacobi_diag(lc)
        coarse = o.PMG(levels=[lc], smoother="jacobi", order=[], bounds=[], lam=[])
        b = lc.mask * o.from_global(lc, wl.random_lvector(lc.n_global, 9))
        dev = torch.device("cuda:0")
        x = torch.empty(lc.gid.size, dtype=torch.float64, device=dev)
        it = se.se_pmg_coarse_solve(P, torch.from_numpy(b.reshape(-1).copy()).to(dev), x)
        xref = o.coarse_solve(coarse, b)
        it_ref = coarse.coarse_iters[-1]
        assert abs(it - it_ref) <= 1
        if it == it_ref:
            assert rel_err(x.cpu().numpy().reshape(lc.gid.shape), xref) <= 1e-8
    finally:
        se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)
