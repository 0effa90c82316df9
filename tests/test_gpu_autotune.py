"""Run-time preconditioner selection (Sec. 5, Table 5): an exhaustive timed search over a small
space of p-multigrid preconditioners on the first solve.

Checks: every candidate is set up and solved to the tolerance (true residual through the
oracle's operator); the chosen one is the fastest converged candidate; the preconditioner handed
back is the chosen one (a solve with it is bit-identical to one with a fresh set-up of the same
description); a space where nothing converges is an error; and the mesh's cached solve graph
never replays with a destroyed preconditioner (the search sets up and destroys one per
candidate, and a new handle may reuse a destroyed one's address).
"""
import math

import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case

pytestmark = pytest.mark.gpu


def rhs(c, k=(1, 2, 1), a=1.3):
    X = c.lv.X
    b = c.empty()
    c.se.se_mesh_rhs(c.m, c.to_gpu(wl.f_rhs_modes(X[0], X[1], X[2], k, a)), b)
    return b


def true_rel_residual(c, b, x):
    bn, xn = c.to_np(b), c.to_np(x)
    r = bn - o.ax(c.lv, xn)
    return math.sqrt(o.dot(c.lv, r, r) / o.dot(c.lv, bn, bn))


@pytest.mark.parametrize("p,precision", [(7, 0), (5, 1)])
def test_search_picks_the_fastest_converged_candidate(p, precision):
    c = Case((3, 3, 3), p, pert=0.05, seed=11)
    se = c.se
    try:
        b = rhs(c)
        cands = se.se_pmg_autotune_space(p, precision)
        assert len(cands) == 3
        best, timed, P = se.se_pmg_autotune(c.m, b, cands, repeats=2, tol=1e-8)
        try:
            assert all(t.status == se.SE_OK for t in timed)
            assert all(t.ms > 0 and t.setup_ms > 0 and t.iterations > 0 for t in timed)
            assert best == min(range(3), key=lambda i: timed[i].ms)
            assert P is not None
            # the handed-back preconditioner is the chosen one
            x1 = c.empty().zero_()
            s1 = se.se_solve(c.m, P, b, x1, tol=1e-8)
            Q = se.se_pmg_setup(c.m, cands[best].pmg)
            x2 = c.empty().zero_()
            s2 = se.se_solve(c.m, Q, b, x2, tol=1e-8)
            se.se_pmg_destroy(Q)
            assert s1.iterations == s2.iterations == timed[best].iterations
            assert c.torch.equal(x1, x2)
            assert true_rel_residual(c, b, x1) <= 2e-8
        finally:
            se.se_pmg_destroy(P)
    finally:
        c.close()


def test_nothing_converges_is_an_error():
    c = Case((2, 2, 2), 5, seed=3)
    se = c.se
    try:
        b = rhs(c)
        cands = se.se_pmg_autotune_space(5)
        with pytest.raises(se.SeError):
            se.se_pmg_autotune(c.m, b, cands, repeats=1, tol=1e-14, maxit=1)
        # the graph solve after a failed search uses only the new preconditioner
        P = se.se_pmg_setup(c.m, cands[1].pmg)
        x = c.empty().zero_()
        st = se.se_solve(c.m, P, b, x, tol=1e-8, graph_capture=1)
        assert true_rel_residual(c, b, x) <= 2e-8 and st.iterations > 0
        se.se_pmg_destroy(P)
    finally:
        c.close()


def test_graph_cache_does_not_outlive_its_preconditioner():
    c = Case((3, 3, 2), 5, seed=5)
    se = c.se
    try:
        b = rhs(c, (2, 1, 1), 0.8)
        ras = se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2)
        jac = se.pmg_desc((5, 3, 1), se.SE_SMOOTH_JACOBI, 1)
        ref = {}
        for name, d in (("ras", ras), ("jac", jac)):
            P = se.se_pmg_setup(c.m, d)
            x = c.empty().zero_()
            ref[name] = (se.se_solve(c.m, P, b, x, tol=1e-9, graph_capture=1).iterations, x.clone())
            se.se_pmg_destroy(P)
        # same b and x buffers every time, so only the preconditioner tells the graphs apart
        x = c.empty()
        for name, d in (("ras", ras), ("jac", jac), ("ras", ras), ("jac", jac)):
            P = se.se_pmg_setup(c.m, d)
            x.zero_()
            st = se.se_solve(c.m, P, b, x, tol=1e-9, graph_capture=1)
            assert st.iterations == ref[name][0], name
            assert c.torch.equal(x, ref[name][1]), name
            se.se_pmg_destroy(P)
    finally:
        c.close()
