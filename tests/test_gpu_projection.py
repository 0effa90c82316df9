"""Projection onto prior solutions (Secs. 3.2 and 4.2, Fischer's method for successive right-hand sides)
and the ||b||-relative stopping rule it is used with.

Checks: a right-hand side in the span of prior ones is solved by the guess alone (0 iterations,
the guess equal to the same combination of prior solutions to the solve tolerance); successive
nearby right-hand sides take fewer iterations with projection than from zero, to the same true
residual (checked with the oracle's operator); the space restarts when full and does not take a
solution it already holds; SE_TOL_B equals SE_TOL_R0 from x0 = 0 (r_0 = b) and stops at once
from an initial guess that already meets the tolerance, in the host loop, the graph solve and
FGMRES.
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, rel_err

pytestmark = pytest.mark.gpu


def setup_case(p=5, nel=(3, 3, 3), schedule=(5, 3, 1), seed=7):
    c = Case(nel, p, pert=0.05, seed=seed)
    P = c.se.se_pmg_setup(c.m, c.se.pmg_desc(schedule, c.se.SE_SMOOTH_RAS, 2))
    return c, P


def rhs_modes(c, k, a):
    X = c.lv.X
    f = wl.f_rhs_modes(X[0], X[1], X[2], k, a)
    b = c.empty()
    c.se.se_mesh_rhs(c.m, c.to_gpu(f), b)
    return b


def true_rel_residual(c, b, x):
    bn, xn = c.to_np(b), c.to_np(x)
    r = bn - o.ax(c.lv, xn)
    return math.sqrt(o.dot(c.lv, r, r) / o.dot(c.lv, bn, bn))


def test_tol_b_matches_tol_r0_from_zero_and_stops_on_a_good_guess():
    c, P = setup_case()
    se, torch = c.se, c.torch
    try:
        b = rhs_modes(c, (1, 2, 1), 1.3)
        for graph in (0, 1):
            x0, x1 = c.empty().zero_(), c.empty().zero_()
            s0 = se.se_solve(c.m, P, b, x0, tol=1e-9, graph_capture=graph)
            s1 = se.se_solve(c.m, P, b, x1, tol=1e-9, graph_capture=graph, tol_norm=se.SE_TOL_B)
            assert s0.iterations == s1.iterations and torch.equal(x0, x1)
            # from the converged solution: already within tol * ||b||
            s2 = se.se_solve(c.m, P, b, x1, tol=1e-8, graph_capture=graph, tol_norm=se.SE_TOL_B)
            assert s2.iterations == 0 and s2.rel_residual <= 1e-8
        x3 = c.empty().zero_()
        s3 = se.se_solve(c.m, P, b, x3, method=se.SE_FGMRES, tol=1e-9, tol_norm=se.SE_TOL_B)
        assert s3.rel_residual <= 1e-9 and true_rel_residual(c, b, x3) <= 2e-9
        s4 = se.se_solve(c.m, P, b, x3, method=se.SE_FGMRES, tol=1e-8, tol_norm=se.SE_TOL_B)
        assert s4.iterations == 0
        with pytest.raises(se.SeError):
            se.se_solve(c.m, P, b, x3, tol=1e-8, tol_norm=7)
    finally:
        c.se.se_pmg_destroy(P)
        c.close()


def test_span_of_prior_right_hand_sides_is_solved_by_the_guess():
    c, P = setup_case()
    se, torch = c.se, c.torch
    proj = se.se_proj_create(c.m, 10)
    try:
        bs = [rhs_modes(c, k, a) for k, a in [((1, 1, 1), 1.0), ((2, 1, 3), 0.7), ((1, 3, 2), 1.9)]]
        xs = []
        for b in bs:
            x = c.empty()
            se.se_proj_guess(proj, b, x)
            st = se.se_solve(c.m, P, b, x, tol=1e-11, tol_norm=se.SE_TOL_B)
            assert st.rel_residual <= 1e-11
            xs.append(x.clone())
            se.se_proj_update(proj, x)
        # a combination of the prior right-hand sides: the guess is the same combination of the
        # prior solutions, and the solve stops at once
        coef = (2.5, -0.4, 1.1)
        b = sum(w * v for w, v in zip(coef, bs))
        xg = c.empty()
        se.se_proj_guess(proj, b, xg)
        ref = sum(w * v for w, v in zip(coef, xs))
        assert rel_err(c.to_np(xg), c.to_np(ref)) <= 1e-8
        st = se.se_solve(c.m, P, b, xg, tol=1e-8, tol_norm=se.SE_TOL_B)
        assert st.iterations == 0
        assert true_rel_residual(c, b, xg) <= 1e-8
    finally:
        se.se_proj_destroy(proj)
        c.se.se_pmg_destroy(P)
        c.close()


def test_successive_right_hand_sides_take_fewer_iterations():
    c, P = setup_case(p=7, nel=(3, 3, 2), schedule=(7, 3, 1), seed=9)
    se = c.se
    proj = se.se_proj_create(c.m, 10)
    try:
        b0 = rhs_modes(c, (1, 1, 1), 1.0)
        db = rhs_modes(c, (2, 3, 1), 1.0)
        cold, warm = [], []
        for step in range(6):
            eps = 0.02 * (step + 1)
            b = b0 + eps * db + (0.5 * eps) ** 2 * rhs_modes(c, (3, 1, 2), 1.0)
            xc = c.empty().zero_()
            cold.append(se.se_solve(c.m, P, b, xc, tol=1e-8, tol_norm=se.SE_TOL_B).iterations)
            xw = c.empty()
            se.se_proj_guess(proj, b, xw)
            st = se.se_solve(c.m, P, b, xw, tol=1e-8, tol_norm=se.SE_TOL_B)
            warm.append(st.iterations)
            assert true_rel_residual(c, b, xw) <= 1.5e-8
            se.se_proj_update(proj, xw)
        assert warm[0] == cold[0]               # empty space: the same solve
        assert sum(warm[3:]) < sum(cold[3:])    # later steps start close to the solution
    finally:
        se.se_proj_destroy(proj)
        c.se.se_pmg_destroy(P)
        c.close()


def test_space_restarts_when_full_and_skips_a_held_solution():
    c, P = setup_case(p=3, nel=(2, 2, 2), schedule=(3, 1))
    se = c.se
    proj = se.se_proj_create(c.m, 2)
    try:
        sizes = []
        xs = []
        for k in [(1, 1, 1), (2, 1, 1), (1, 2, 1)]:
            b = rhs_modes(c, k, 1.0)
            x = c.empty().zero_()
            se.se_solve(c.m, P, b, x, tol=1e-10)
            xs.append(x)
            sizes.append(se.se_proj_update(proj, x))
        assert sizes == [1, 2, 1]               # third update restarts the full space
        assert se.se_proj_update(proj, 3.0 * xs[2]) == 1  # a multiple of the held vector
        with pytest.raises(se.SeError):
            se.se_proj_create(c.m, 0)
    finally:
        se.se_proj_destroy(proj)
        c.se.se_pmg_destroy(P)
        c.close()


def test_guess_equals_the_oracle_projection():
    """se_proj_guess against the oracle's A-orthogonal projection of A^-1 b onto the span of the
    prior solutions (its plain definition, a Galerkin solve), for arbitrary prior vectors and a
    right-hand side outside their span: 1e-9 relative."""
    c, P = setup_case(p=5, nel=(3, 2, 2), schedule=(5, 3, 1), seed=3)
    se = c.se
    proj = se.se_proj_create(c.m, 6)
    try:
        xs = [c.random_continuous(100 + k) for k in range(4)]
        for x in xs:
            se.se_proj_update(proj, c.to_gpu(x))
        b = o.ax(c.lv, c.random_continuous(200))
        g = c.empty()
        se.se_proj_guess(proj, c.to_gpu(b), g)
        ref = o.projection_guess(c.lv, xs, b)
        assert rel_err(c.to_np(g), ref) <= 1e-9
    finally:
        se.se_proj_destroy(proj)
        c.se.se_pmg_destroy(P)
        c.close()
