"""GPU parity of whole solves (Sec. 2.2 outer Krylov with the Sec. 2.2 preconditioners).

Bar: the GPU solution meets the requested relative residual 1e-8 (checked with the ORACLE's
operator on the GPU solution), and its iteration count is within +-1 of the oracle's on the
same seeded problem.  Mixed precision (FP32 preconditioner): residual 1e-8 reached; the error
against the FP64 oracle solution and the iteration counts are reported.
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, rel_err

pytestmark = pytest.mark.gpu


def gpu_problem(c):
    xyz = c.empty(3 * c.info.L)
    c.se.se_mesh_nodes(c.m, xyz)
    X = xyz.cpu().numpy().reshape(3, -1)
    f = wl.f_rhs(X[0], X[1], X[2])
    b = c.empty()
    c.se.se_mesh_rhs(c.m, c.to_gpu(f), b)
    return b


def true_rel_residual(c, x_np, b_np):
    r = b_np - o.ax(c.lv, x_np)
    return math.sqrt(o.dot(c.lv, r, r) / o.dot(c.lv, b_np, b_np))


SMALL = dict(nel=(4, 4, 4), p=7, pert=0.0)


@pytest.mark.parametrize("pre,method", [("jacobi", "fpcg"), ("ras", "fpcg"), ("ras", "fgmres"),
                                        ("chebjac", "fpcg"), ("asm", "fpcg")])
def test_small_box_solve_parity(pre, method):
    c = Case(SMALL["nel"], SMALL["p"], pert=SMALL["pert"])
    se = c.se
    P = None
    try:
        b = gpu_problem(c)
        lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
        assert rel_err(c.to_np(b), bo) <= 1e-13
        if pre == "jacobi":
            pmg = None
        else:
            sm = {"ras": "ras", "asm": "asm", "chebjac": "jacobi"}[pre]
            P = se.se_pmg_setup(c.m, se.pmg_desc((7, 3, 1), {"ras": 1, "asm": 2, "jacobi": 0}[sm], 2))
            pmg = o.pmg_setup(c.V, c.nel, (7, 3, 1), smoother=sm, order=2, amp=c.amp)
        x = c.empty().zero_()
        meth = se.SE_FPCG if method == "fpcg" else se.SE_FGMRES
        st = se.se_solve(c.m, P, b, x, method=meth, tol=1e-8, maxit=2000, restart=20)
        xo, it_o, rel_o = o.solve(lvo, bo, pmg, method=method, tol=1e-8, maxit=2000)
        assert st.rel_residual <= 1e-8
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        assert true_rel_residual(c, c.to_np(x), bo) <= 1.5e-8
        assert rel_err(c.to_np(x), xo) <= 1e-5
        print(f"{pre}/{method}: gpu {st.iterations} it, oracle {it_o} it, {st.ms_total:.1f} ms")
    finally:
        if P:
            se.se_pmg_destroy(P)
        c.close()


@pytest.mark.parametrize("p,schedule", [(7, (7, 3, 1)), (9, (9, 5, 1)), (9, (9, 7, 5, 1))])
def test_mixed_precision_solve(p, schedule):
    c = Case((4, 4, 4), p, pert=0.0)
    se = c.se
    P64 = P32 = None
    try:
        b = gpu_problem(c)
        P64 = se.se_pmg_setup(c.m, se.pmg_desc(schedule, se.SE_SMOOTH_RAS, 2, precision=se.SE_FP64))
        P32 = se.se_pmg_setup(c.m, se.pmg_desc(schedule, se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32))
        x64, x32 = c.empty().zero_(), c.empty().zero_()
        s64 = se.se_solve(c.m, P64, b, x64, tol=1e-8)
        s32 = se.se_solve(c.m, P32, b, x32, tol=1e-8)
        lvo, bo = o.problem(c.V, c.nel, p, amp=c.amp)
        pmg = o.pmg_setup(c.V, c.nel, schedule, smoother="ras", order=2, amp=c.amp)
        xo, it_o, _ = o.solve(lvo, bo, pmg, tol=1e-8)
        assert abs(s64.iterations - it_o) <= 1
        assert true_rel_residual(c, c.to_np(x32), bo) <= 1.5e-8
        err32 = rel_err(c.to_np(x32), xo)
        assert err32 <= 1e-5
        assert s32.iterations <= s64.iterations + 3
        u_star = wl.u_exact(*lvo.X)
        print(f"p={p} {schedule}: fp64 {s64.iterations} it, fp32-precond {s32.iterations} it, "
              f"oracle {it_o} it, |x32-x_oracle|/|x| {err32:.2e}, "
              f"|x32-u*| {np.max(np.abs(c.to_np(x32) - u_star)):.2e}")
    finally:
        for P in (P64, P32):
            if P:
                se.se_pmg_destroy(P)
        c.close()


def test_solve_reuses_mesh_and_is_deterministic():
    c = Case((3, 3, 3), 5, pert=0.05, seed=4)
    se = c.se
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 1))
    try:
        b = gpu_problem(c)
        x1, x2 = c.empty().zero_(), c.empty().zero_()
        s1 = se.se_solve(c.m, P, b, x1, tol=1e-10)
        s2 = se.se_solve(c.m, P, b, x2, tol=1e-10)
        assert s1.iterations == s2.iterations
        assert c.torch.equal(x1, x2)
        # a warm start: the tolerance is relative to the warm start's own residual
        x3 = x1.clone()
        s3 = se.se_solve(c.m, P, b, x3, tol=1e-4)
        assert s3.iterations < s1.iterations
        assert float((x3 - x1).abs().max()) <= 1e-8 * float(x1.abs().max())
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_not_converged_status():
    c = Case((3, 3, 3), 5)
    se = c.se
    try:
        b = gpu_problem(c)
        x = c.empty().zero_()
        with pytest.raises(se.SeError) as e:
            se.se_solve(c.m, None, b, x, tol=1e-12, maxit=3)
        assert e.value.code == se.SE_ENOTCONV
        st = se.se_solve(c.m, None, b, x.zero_(), tol=1e-12, maxit=3, allow_notconv=True)
        assert st.iterations == 3 and st.status == se.SE_ENOTCONV
    finally:
        c.close()


def test_injected_allocation_failures_leave_the_library_usable():
    """Host-side fault injection (no device fault): se_selftest_fail_alloc(n) makes the n-th
    following device allocation fail with SE_ENOMEM before any CUDA call.  Sweeping n over every
    allocation of a mesh set-up, an FP32-V-cycle preconditioner set-up and a first graph solve,
    each run fails with SE_ENOMEM from the call that allocates (the handles it built are freed),
    and afterwards the library builds and solves the same problem to the same bits."""
    torch, se = Case((1, 1, 1), 1).torch, Case((1, 1, 1), 1).se
    nel, p = (2, 2, 2), 5
    V = wl.vertex_lattice(nel, 0.05, seed=1)

    def run():
        m = se.se_mesh_create(nel, p, vertex_xyz=V, deform_amp=wl.DEFORM_AMP)
        P = None
        try:
            L = se.se_mesh_get_info(m).L
            xyz = torch.empty(3 * L, dtype=torch.float64, device="cuda")
            se.se_mesh_nodes(m, xyz)
            X = xyz.cpu().numpy().reshape(3, -1)
            b = torch.empty(L, dtype=torch.float64, device="cuda")
            se.se_mesh_rhs(m, torch.from_numpy(wl.f_rhs(X[0], X[1], X[2])).cuda(), b)
            P = se.se_pmg_setup(m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32))
            x = torch.zeros_like(b)
            st = se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1)
            return x.cpu().numpy(), st.iterations
        finally:
            if P:
                se.se_pmg_destroy(P)
            se.se_mesh_destroy(m)

    ref, it_ref = run()
    failures = 0
    for n in range(1, 500):
        se.se_selftest_fail_alloc(n)
        try:
            run()
        except se.SeError as e:
            assert e.code == se.SE_ENOMEM, (n, str(e))
            failures += 1
            continue
        finally:
            se.se_selftest_fail_alloc(0)
        break  # n is past the sequence's last allocation: the run completed
    assert failures >= 20, failures
    x, it = run()
    assert it == it_ref and np.array_equal(x, ref)
    with pytest.raises(se.SeError):
        se.se_selftest_fail_alloc(-1)


@pytest.mark.parametrize("method", ["fpcg", "fgmres"])
@pytest.mark.parametrize("graph", [0, 1])
def test_degenerate_problems(method, graph):
    """Zero right-hand side (the solution is x = 0: no iteration, no division by the zero initial
    residual), a mesh whose every node is on the Dirichlet boundary (no unknown at all: one
    element, p = 1) and one with a single unknown (one element, p = 2, pMG 2-1)."""
    c = Case((2, 2, 1), 5, seed=4)
    se = c.se
    meth = se.SE_FPCG if method == "fpcg" else se.SE_FGMRES
    if graph and method == "fgmres":
        pytest.skip("the graph solve is FPCG")
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2))
    try:
        b = c.empty().zero_()
        x = c.empty().zero_()
        st = se.se_solve(c.m, P, b, x, method=meth, tol=1e-8, graph_capture=graph)
        assert st.iterations == 0 and st.rel_residual == 0.0
        assert float(x.abs().max()) == 0.0
    finally:
        se.se_pmg_destroy(P)
        c.close()
    for nel, p, sched in [((1, 1, 1), 1, None), ((1, 1, 1), 2, (2, 1))]:
        c = Case(nel, p, seed=5)
        P = se.se_pmg_setup(c.m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 2)) if sched else None
        try:
            xyz = c.empty(3 * c.info.L)
            se.se_mesh_nodes(c.m, xyz)
            X = xyz.cpu().numpy().reshape(3, -1)
            b = c.empty()
            se.se_mesh_rhs(c.m, c.to_gpu(wl.f_rhs(X[0], X[1], X[2])), b)
            x = c.empty().zero_()
            st = se.se_solve(c.m, P, b, x, method=meth, tol=1e-8, graph_capture=graph)
            lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
            if np.max(np.abs(bo)) == 0.0:  # no unknown: nothing to solve
                assert st.iterations == 0 and float(x.abs().max()) == 0.0
            else:
                xo, it_o, _ = o.solve(lvo, bo, o.pmg_setup(c.V, nel, sched, smoother="ras", order=2,
                                                          amp=c.amp) if sched else None,
                                      method=method, tol=1e-8)
                assert st.rel_residual <= 1e-8 and rel_err(c.to_np(x), xo) <= 1e-8
        finally:
            if P:
                se.se_pmg_destroy(P)
            c.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_headline_configuration_against_the_oracle(graph):
    """The benchmark's own solve on a smaller piece of its workload: 6^3 elements of the map
    with the interior lattice vertices perturbed by up to 5% of h (seed 0, the library's
    generator), p = 7, pMG 7-5-3-1 with Chebyshev-Jacobi order 1 on every smoothed level
    (Algorithms 1-2), coarse Jacobi-PCG, FPCG to 1e-8, host-driven and as one graph launch.
    Iterations within one of the oracle's; true residual and solution checked with the
    oracle's operator and solution."""
    from tests.gpu_common import gpu
    torch, se = gpu()
    nel, p, sched = (6, 6, 6), 7, (7, 5, 3, 1)
    m = se.se_mesh_create(nel, p, perturb_frac=0.05, seed=0, deform_amp=wl.DEFORM_AMP)
    P = None
    try:
        V = wl.vertex_lattice(nel, 0.05, seed=0)
        Vg = np.empty(V.size)
        se.se_mesh_vertices(m, Vg)
        assert np.array_equal(Vg, V.reshape(-1))
        info = se.se_mesh_get_info(m)
        dev = torch.device("cuda:0")
        xyz = torch.empty(3 * info.L, dtype=torch.float64, device=dev)
        se.se_mesh_nodes(m, xyz)
        X = xyz.cpu().numpy().reshape(3, -1)
        b = torch.empty(info.L, dtype=torch.float64, device=dev)
        se.se_mesh_rhs(m, torch.from_numpy(wl.f_rhs(X[0], X[1], X[2])).to(dev), b)
        P = se.se_pmg_setup(m, se.pmg_desc(sched, se.SE_SMOOTH_JACOBI, 1))
        x = torch.zeros_like(b)
        st = se.se_solve(m, P, b, x, method=se.SE_FPCG, tol=1e-8, graph_capture=graph)
        lvo, bo = o.problem(V, nel, p, amp=wl.DEFORM_AMP)
        pmg = o.pmg_setup(V, nel, sched, smoother="jacobi", order=1, amp=wl.DEFORM_AMP)
        for l in range(len(sched) - 1):
            lam = se.se_pmg_lambda(P, l)
            assert abs(lam - pmg.lam[l]) <= 1e-9 * pmg.lam[l]
        xo, it_o, _ = o.solve(lvo, bo, pmg, tol=1e-8)
        xg = x.cpu().numpy().reshape(xo.shape)
        assert np.max(np.abs(b.cpu().numpy().reshape(bo.shape) - bo)) <= 1e-13 * np.max(np.abs(bo))
        assert st.rel_residual <= 1e-8
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        r = bo - o.ax(lvo, xg)
        assert math.sqrt(o.dot(lvo, r, r) / o.dot(lvo, bo, bo)) <= 1.5e-8
        assert rel_err(xg, xo) <= 1e-6
        print(f"headline config 6^3 (graph={graph}): gpu {st.iterations} it, oracle {it_o} it, "
              f"max rel diff {rel_err(xg, xo):.2e}")
    finally:
        if P:
            se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)


@pytest.mark.parametrize("graph", [0, 1])
def test_solve_with_host_buffers_equals_the_device_solve(graph):
    """se_solve_host (b copied in, x from zero or from a host guess, x copied out inside the call)
    gives bitwise the device solve's result and statistics, with pinned and with pageable host
    buffers; a repeated call reuses the mesh's device vectors (and, graph-driven, its graph)."""
    c = Case((4, 3, 3), 5, seed=8)
    se, torch = c.se, c.torch
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_JACOBI, 1))
    try:
        b = c.to_gpu(c.random_continuous(31))
        x = torch.zeros_like(b)
        ref = se.se_solve(c.m, P, b, x, tol=1e-8, graph_capture=graph)
        xref = x.cpu().numpy()
        for pinned in (False, True):
            bh = b.cpu()
            xh = torch.full((c.info.L,), float("nan"), dtype=torch.float64)
            if pinned:
                bh, xh = bh.pin_memory(), xh.pin_memory()
            for _ in range(2):
                st = se.se_solve_host(c.m, P, bh, xh, tol=1e-8, graph_capture=graph)
                assert st.iterations == ref.iterations and st.rel_residual == ref.rel_residual
                assert np.array_equal(xh.numpy(), xref)
        # from a host initial guess: the solve with that guess on the device
        x0 = c.random_continuous(32)
        x.copy_(c.to_gpu(x0))
        ref0 = se.se_solve(c.m, P, b, x, tol=1e-8, graph_capture=graph)
        xh = np.empty(c.info.L)
        st0 = se.se_solve_host(c.m, P, b.cpu().numpy(), xh, x0_host=np.ascontiguousarray(x0.reshape(-1)),
                               tol=1e-8, graph_capture=graph)
        assert st0.iterations == ref0.iterations
        assert np.array_equal(xh, x.cpu().numpy())
        with pytest.raises(ValueError):
            se.se_solve_host(c.m, P, b, xh)   # a device tensor is not a host buffer
    finally:
        se.se_pmg_destroy(P)
        c.close()
