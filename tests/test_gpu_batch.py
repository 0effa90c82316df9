"""Device-driven solves (one CUDA graph per solve) and batched solves (one graph for many).

The graph solve runs the same kernels as the host-driven loop with the same arithmetic per
point, so iterations and solutions must agree exactly.  In a batch, problems that share a
preconditioner configuration are solved as one union problem per group: each must meet the
tolerance (checked with the library's FP64 operator) and agree with its stand-alone solve to
within rounding; problems that run alone in the batch graph must equal their stand-alone solve
bitwise; and the batch must be deterministic (two runs, the same bits).
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, gpu, rel_err

pytestmark = pytest.mark.gpu


def problem(se, torch, nel, p, seed, schedule, precision, smoother=1):
    m = se.se_mesh_create(nel, p, perturb_frac=0.05, seed=seed, deform_amp=wl.DEFORM_AMP)
    info = se.se_mesh_get_info(m)
    xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, -1).cpu().numpy()
    k, a = wl.request_modes(seed)
    f = torch.from_numpy(wl.f_rhs_modes(X[0], X[1], X[2], k, a)).cuda()
    b = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_rhs(m, f, b)
    P = se.se_pmg_setup(m, se.pmg_desc(schedule, smoother, 2, precision=precision))
    return m, P, b, info


@pytest.mark.parametrize("pre", ["ras", "jacobi_pcg"])
def test_graph_solve_equals_host_loop(pre):
    torch, se = gpu()
    m, P, b, info = problem(se, torch, (4, 3, 3), 7, 3, (7, 3, 1), se.SE_FP64)
    try:
        Pu = P if pre == "ras" else None
        x1 = torch.zeros_like(b)
        x2 = torch.zeros_like(b)
        s1 = se.se_solve(m, Pu, b, x1, tol=1e-9)
        s2 = se.se_solve(m, Pu, b, x2, tol=1e-9, graph_capture=1)
        assert s1.iterations == s2.iterations
        assert abs(s1.rel_residual - s2.rel_residual) <= 1e-12
        assert rel_err(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-14
        # replay the cached graph: same result again
        x2.zero_()
        s3 = se.se_solve(m, Pu, b, x2, tol=1e-9, graph_capture=1)
        assert s3.iterations == s1.iterations
        assert rel_err(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-14
    finally:
        se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)


def true_rel_residual(se, torch, m, b, x):
    """||b - A x|| / ||b|| with the library's FP64 operator and unique-node inner products."""
    r = torch.empty_like(b)
    se.se_residual(m, b, x, r, 0)
    return math.sqrt(se.se_dot(m, r, r) / se.se_dot(m, b, b))


def test_batch_groups_match_alone_and_converge():
    """Problems sharing a preconditioner configuration are solved as one union problem per
    group (one launch per phase for all members); the rest run alone in the same graph.
    Every problem meets the tolerance; grouped ones agree with their stand-alone solves to
    within rounding (iterations within one), alone ones bitwise; the batch is deterministic."""
    torch, se = gpu()
    specs = [((4, 4, 4), 3, (3, 1), se.SE_FP32, 1), ((3, 4, 4), 3, (3, 1), se.SE_FP32, 1),
             ((5, 4, 3), 5, (5, 3, 1), se.SE_FP32, 1), ((3, 3, 4), 7, (7, 3, 1), se.SE_FP32, 1),
             ((4, 3, 3), 7, (7, 3, 1), se.SE_FP32, 1), ((3, 3, 3), 9, (9, 5, 1), se.SE_FP32, 1),
             ((4, 4, 4), 7, (7, 5, 3, 1), se.SE_FP64, 1), ((3, 4, 3), 7, (7, 5, 3, 1), se.SE_FP64, 1),
             ((4, 3, 4), 5, (5, 3, 1), se.SE_FP64, 0), ((3, 3, 3), 5, (5, 3, 1), se.SE_FP64, 0),
             ((3, 3, 3), 7, (7, 3, 1), se.SE_FP32, 2)]
    specs.insert(2, ((1, 3, 4), 3, (3, 1), se.SE_FP32, 1))
    probs = [problem(se, torch, nel, p, 40 + i, sch, prec, sm)
             for i, (nel, p, sch, prec, sm) in enumerate(specs)]
    # one problem without a preconditioner (Jacobi PCG): runs alone
    mj, Pj, bj, _ = problem(se, torch, (3, 3, 3), 3, 77, (3, 1), se.SE_FP64)
    try:
        entries = [(m, P, b) for (m, P, b, _) in probs] + [(mj, None, bj)]
        alone = []
        for m, P, b in entries:
            x = torch.zeros_like(b)
            st = se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1)
            alone.append((st.iterations, x.clone()))
        xs = [torch.zeros_like(b) for (_, _, b) in entries]
        B = se.se_batch_create([(m, P, b, x) for (m, P, b), x in zip(entries, xs)], tol=1e-8)
        try:
            groups, grouped = se.se_batch_info(B)
            # FP32 RAS p=3 (3, one member a single element row), p=7 7-3-1 (2), FP64 RAS 7-5-3-1
            # (2), FP64 Jacobi p=5 (2), and the single-member groups of p=5 and p=9; ASM and no
            # preconditioner run alone
            assert groups == 6 and grouped == 11, (groups, grouped)
            first = None
            for rep in range(2):
                for x in xs:
                    x.zero_()
                se.se_batch_run(B)
                stats = se.se_batch_stats(B, len(entries))
                got = [x.clone() for x in xs]
                for k, ((it, xa), st, x, (m, P, b)) in enumerate(zip(alone, stats, xs, entries)):
                    assert st.rel_residual <= 1e-8, (k, st.rel_residual)
                    assert true_rel_residual(se, torch, m, b, x) <= 1.5e-8, k
                    if k >= 11:   # alone in the graph: the se_solve graph itself
                        assert st.iterations == it and torch.equal(x, xa), k
                    else:
                        assert abs(st.iterations - it) <= 1, (k, st.iterations, it)
                        err = float((x - xa).abs().max() / xa.abs().max())
                        assert err <= 1e-6, (k, err)
                if first is None:
                    first = (got, [s.iterations for s in stats])
                else:
                    assert [s.iterations for s in stats] == first[1]
                    assert all(torch.equal(a, b_) for a, b_ in zip(got, first[0]))
        finally:
            se.se_batch_destroy(B)
        # one-call form
        for x in xs:
            x.zero_()
        stats = se.se_batch_solve([(m, P, b, x) for (m, P, b), x in zip(entries, xs)], tol=1e-8)
        assert [s.iterations for s in stats] == first[1]
    finally:
        for m, P, b, info in probs:
            se.se_pmg_destroy(P)
            se.se_mesh_destroy(m)
        se.se_pmg_destroy(Pj)
        se.se_mesh_destroy(mj)


def test_batch_group_tolerance_relative_to_b():
    """The ||b||-relative stopping rule per member of a group, from a non-zero initial guess."""
    torch, se = gpu()
    probs = [problem(se, torch, nel, 5, 60 + i, (5, 3, 1), se.SE_FP32)
             for i, nel in enumerate([(3, 3, 3), (4, 3, 3), (3, 4, 3)])]
    try:
        xs = []
        for m, P, b, info in probs:
            x = torch.zeros_like(b)
            se.se_solve(m, P, b, x, tol=1e-3, graph_capture=1)   # a rough initial guess
            xs.append(x)
        stats = se.se_batch_solve([(m, P, b, x) for (m, P, b, _), x in zip(probs, xs)], tol=1e-9,
                                  tol_norm=se.SE_TOL_B)
        for (m, P, b, _), x, st in zip(probs, xs, stats):
            assert st.rel_residual <= 1e-9
            assert true_rel_residual(se, torch, m, b, x) <= 2e-9
    finally:
        for m, P, b, info in probs:
            se.se_pmg_destroy(P)
            se.se_mesh_destroy(m)


def test_batch_problem_matches_oracle():
    c = Case((3, 3, 3), 5, pert=0.05, seed=12)
    se, torch = c.se, c.torch
    P = se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2))
    try:
        f = wl.f_rhs(*c.lv.X)
        b = c.empty()
        se.se_mesh_rhs(c.m, c.to_gpu(f), b)
        x = c.empty().zero_()
        st = se.se_batch_solve([(c.m, P, b, x)], tol=1e-8)[0]
        lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
        pmg = o.pmg_setup(c.V, c.nel, (5, 3, 1), smoother="ras", order=2, amp=c.amp)
        xo, it_o, _ = o.solve(lvo, bo, pmg, tol=1e-8)
        assert abs(st.iterations - it_o) <= 1
        r = bo - o.ax(lvo, c.to_np(x))
        assert math.sqrt(o.dot(lvo, r, r) / o.dot(lvo, bo, bo)) <= 1.5e-8
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_batch_rejects_shared_mesh():
    torch, se = gpu()
    m, P, b, info = problem(se, torch, (2, 2, 2), 3, 1, (3, 1), se.SE_FP64)
    try:
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        with pytest.raises(se.SeError) as e:
            se.se_batch_create([(m, P, b, x1), (m, P, b, x2)])
        assert e.value.code == se.SE_EINVAL
    finally:
        se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)


def test_batch_size_classes_form_separate_groups():
    """Problems of one preconditioner configuration whose element counts fall in different size
    classes (below 4096 elements, then one class per factor 8) are solved as different groups,
    each converging as its stand-alone solve does."""
    torch, se = gpu()
    specs = [((4, 4, 4), 3, 61), ((5, 4, 4), 3, 62), ((16, 16, 16), 3, 63)]
    probs = [problem(se, torch, nel, p, seed, (3, 1), se.SE_FP32) for nel, p, seed in specs]
    try:
        entries = [(m, P, b) for (m, P, b, _) in probs]
        alone = []
        for m, P, b in entries:
            x = torch.zeros_like(b)
            alone.append(se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1).iterations)
        xs = [torch.zeros_like(b) for (_, _, b) in entries]
        B = se.se_batch_create([(m, P, b, x) for (m, P, b), x in zip(entries, xs)], tol=1e-8)
        try:
            assert se.se_batch_info(B) == (2, 3)
            se.se_batch_run(B)
            stats = se.se_batch_stats(B, len(entries))
            for k, (st, x, (m, P, b)) in enumerate(zip(stats, xs, entries)):
                assert abs(st.iterations - alone[k]) <= 1, k
                assert true_rel_residual(se, torch, m, b, x) <= 1.5e-8, k
        finally:
            se.se_batch_destroy(B)
    finally:
        for m, P, b, _ in probs:
            se.se_pmg_destroy(P)
            se.se_mesh_destroy(m)
