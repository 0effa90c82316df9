"""Pins of the oracle's smoothers, multigrid and Krylov solvers (CPU only).

FDM / Schwarz: on rectilinear (tensor-product) box meshes the separable extended operator of
eq 5 is exactly the Galerkin restriction R_e A R_e^T, so the fast-diagonalisation solve of eqs
8-9 must equal the dense inverse of that window of the brute-force assembled matrix.
Chebyshev (Algorithm 2): I - M A equals the scaled Chebyshev polynomial of SA, built here by the
three-term recurrence and cosh(m arccosh sigma).  Arnoldi: exact once the Krylov space is
exhausted.  Multigrid: the transfers are adjoint and reproduce coarse polynomials; the V-cycle
(Algorithm 1) with an exact coarse solve equals the product of the error propagators of its
steps (pre-smoothing, coarse correction with the re-evaluated residual, post-smoothing) built
from dense matrices, and contracts the error.  Solvers: the converged solution equals a dense
direct solve; the discrete solution converges spectrally; flexible CG reduces to textbook PCG
for a fixed preconditioner and keeps consecutive directions conjugate for a varying one;
FGMRES reaches the minimal residual over its Krylov space (and per restart cycle).
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.dense_reference import assembled_stiffness, free_nodes


def rectilinear_lattice(xs, ys, zs):
    V = np.empty((len(zs), len(ys), len(xs), 3))
    V[..., 0] = np.asarray(xs)[None, None, :]
    V[..., 1] = np.asarray(ys)[None, :, None]
    V[..., 2] = np.asarray(zs)[:, None, None]
    return V


def window_nodes(lv, e):
    """Global ids of the free nodes of element e's extended window, in window order, and their
    positions (a, b, c) in the pbar^3 window."""
    p = lv.p
    pb = p + 3
    nx, ny, nz = lv.nel
    NX, NY, NZ = lv.lattice
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    free = np.zeros(lv.n_global, dtype=bool)
    free[lv.gid[lv.mask > 0]] = True
    ids, pos = [], []
    for c in range(pb):
        for b in range(pb):
            for a in range(pb):
                I, J, K = ex * p - 1 + a, ey * p - 1 + b, ez * p - 1 + c
                if 0 <= I < NX and 0 <= J < NY and 0 <= K < NZ:
                    g = I + NX * (J + NY * K)
                    if free[g]:
                        ids.append(g)
                        pos.append((c, b, a))
    return np.array(ids), pos


@pytest.fixture(scope="module", params=[("D",) * 6, ("N", "D", "D", "N", "D", "D")])
def rect_case(request):
    V = rectilinear_lattice([0, 0.3, 0.55, 1.0], [0, 0.45, 1.0], [0, 0.6, 1.0])
    nel = (3, 2, 2)
    p = 3
    lv = o.make_level(V, nel, p, bc=request.param, amp=0.0)
    x, w = o.gll(p)
    A = assembled_stiffness(lv, x, w)
    lv.extra["fdm"] = o.fdm_setup(lv, V, amp=0.0)
    return V, lv, A


def test_fdm_similarity_transforms():
    rng = np.random.default_rng(0)
    for p in (3, 5, 7):
        for hl, hr, dl, dr in [(True, True, True, True), (False, True, True, True),
                               (True, False, True, True), (False, True, False, True)]:
            lens = rng.uniform(0.5, 2.0, size=(4, 3))
            Ab, Bd, active = o.fdm_1d(p, lens, hl, hr, dl, dr)
            S, L = o.fdm_factors(p, lens, hl, hr, dl, dr)
            Sa = S[:, active, :len(active)]
            for m in range(4):
                StAS = Sa[m].T @ Ab[m] @ Sa[m]
                StBS = Sa[m].T @ np.diag(Bd[m]) @ Sa[m]
                assert np.allclose(StAS, np.diag(L[m, :len(active)]), atol=1e-12 * np.abs(StAS).max())
                assert np.allclose(StBS, np.eye(len(active)), atol=1e-13)
            assert Ab.shape[1] == (p + 3) - (not hl) - (not hr) - ((not hl) and dl) - ((not hr) and dr)


def test_fdm_equals_dense_window_inverse(rect_case):
    V, lv, A = rect_case
    S, Lm = lv.extra["fdm"]
    rng = np.random.default_rng(1)
    pb = lv.p + 3
    for e in range(lv.E):
        ids, pos = window_nodes(lv, e)
        Aw = A[np.ix_(ids, ids)]
        rw = rng.standard_normal(len(ids))
        rbar = np.zeros((1, pb, pb, pb))
        for v, (c, b, a) in zip(rw, pos):
            rbar[0, c, b, a] = v
        z = o.fdm_apply(S[e:e + 1], Lm[e:e + 1], rbar)[0]
        zw = np.array([z[c, b, a] for (c, b, a) in pos])
        assert np.allclose(zw, np.linalg.solve(Aw, rw), rtol=1e-11, atol=1e-11 * np.abs(zw).max())
        inactive = np.ones((pb, pb, pb), dtype=bool)
        for (c, b, a) in pos:
            inactive[c, b, a] = False
        assert np.all(z[inactive] == 0.0)


def dense_schwarz(lv, A, kind):
    """Dense RAS (own nodes weighted 1/mult) or ASM (whole window, then divided by the
    number of windows covering the node) with exact window inverses."""
    n = lv.n_global
    Msum = np.zeros((n, n))
    cover = np.zeros(n)
    mult_g = np.zeros(n)
    mult_g[lv.gid.ravel()] = lv.mult.ravel()
    for e in range(lv.E):
        ids, pos = window_nodes(lv, e)
        inv = np.linalg.inv(A[np.ix_(ids, ids)])
        own = set(lv.gid[e].ravel().tolist())
        for r_, g in enumerate(ids):
            if kind == "ras":
                if g in own:
                    Msum[g, ids] += inv[r_] / mult_g[g]
            else:
                Msum[g, ids] += inv[r_]
                cover[g] += 1
    if kind == "asm":
        nz = cover > 0
        Msum[nz] /= cover[nz][:, None]
    return Msum


@pytest.mark.parametrize("kind", ["ras", "asm"])
def test_schwarz_equals_dense(rect_case, kind):
    V, lv, A = rect_case
    M = dense_schwarz(lv, A, kind)
    rng = np.random.default_rng(2)
    rg = rng.standard_normal(lv.n_global)
    r = lv.mask * o.from_global(lv, rg)
    s = o.ras(lv, r) if kind == "ras" else o.asm(lv, r)
    cols = free_nodes(lv)
    ref = M[np.ix_(cols, cols)] @ o.to_global(lv, r)[cols]
    assert np.allclose(o.to_global(lv, s)[cols], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def chebyshev_matrix_polynomial(SA, lmin, lmax, m):
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    X = (theta * np.eye(len(SA)) - SA) / delta
    T0, T1 = np.eye(len(SA)), X
    for _ in range(m - 1):
        T0, T1 = T1, 2 * X @ T1 - T0
    sigma = theta / delta
    return T1 / math.cosh(m * math.acosh(sigma))


def operator_matrix(lv, fn, cols):
    M = np.zeros((len(cols), len(cols)))
    for n, g in enumerate(cols):
        ug = np.zeros(lv.n_global)
        ug[g] = 1.0
        M[:, n] = o.to_global(lv, fn(lv.mask * o.from_global(lv, ug)))[cols]
    return M


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("smoother", ["jacobi", "ras"])
def test_chebyshev_error_operator(rect_case, order, smoother):
    V, lv, A = rect_case
    lv.extra["diag"] = o.jacobi_diag(lv)
    cols = free_nodes(lv)
    Af = A[np.ix_(cols, cols)]
    S = (lambda r: o.jacobi(lv, r)) if smoother == "jacobi" else (lambda r: o.ras(lv, r))
    Sm = operator_matrix(lv, S, cols)
    SA = Sm @ Af
    lmax_true = np.max(np.abs(np.linalg.eigvals(SA)))
    lmin, lmax = 0.1 * lmax_true, 1.1 * lmax_true
    Mm = operator_matrix(lv, lambda r: o.chebyshev(r, lambda u: o.ax(lv, u), S, lmin, lmax, order), cols)
    lhs = np.eye(len(cols)) - Mm @ Af
    rhs_ = chebyshev_matrix_polynomial(SA, lmin, lmax, order + 1)
    assert np.allclose(lhs, rhs_, atol=1e-9)
    if smoother == "jacobi":
        # SA is similar to an SPD matrix: on [lmin, lmax] the amplification is bounded by
        # 1/T_{k+1}(sigma); below lmin it stays below 1
        ev = np.linalg.eigvals(SA).real
        theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
        bound = 1.0 / math.cosh((order + 1) * math.acosh(theta / delta))
        amp = np.abs(np.linalg.eigvals(lhs))
        inside = (ev >= lmin) & (ev <= lmax)
        amp_in = np.abs(np.polynomial.chebyshev.chebval((theta - ev[inside]) / delta, [0] * (order + 1) + [1])) * bound
        assert np.all(amp_in <= bound * (1 + 1e-9))
        assert amp.max() <= 1.0 + 1e-9


@pytest.mark.parametrize("smoother", ["jacobi", "ras"])
def test_arnoldi_estimate(rect_case, smoother):
    V, lv, A = rect_case
    lv.extra["diag"] = o.jacobi_diag(lv)
    cols = free_nodes(lv)
    S = (lambda r: o.jacobi(lv, r)) if smoother == "jacobi" else (lambda r: o.ras(lv, r))
    SA = operator_matrix(lv, S, cols) @ A[np.ix_(cols, cols)]
    lam_true = np.max(np.abs(np.linalg.eigvals(SA)))
    v0 = lv.mask * o.from_global(lv, wl.arnoldi_start_global(1000, lv.n_global))
    dotf = lambda a, b: o.dot(lv, a, b)
    Aop = lambda u: o.ax(lv, u)
    lam_full, _ = o.arnoldi_lambda(Aop, S, v0, dotf, steps=len(cols) + 5)
    assert abs(lam_full - lam_true) < 1e-9 * lam_true
    lam10, H = o.arnoldi_lambda(Aop, S, v0, dotf, steps=10)
    assert H.shape == (11, 10)
    assert 0.8 * lam_true < lam10 <= lam_true * (1 + 1e-10)


@pytest.fixture(scope="module")
def mg_case():
    nel = (2, 2, 2)
    V = wl.vertex_lattice(nel, 0.1, seed=4)
    return V, nel


def test_transfers_adjoint_and_exact(mg_case):
    V, nel = mg_case
    for pf, pc in [(5, 3), (3, 1), (7, 3)]:
        lf = o.make_level(V, nel, pf)
        lc = o.make_level(V, nel, pc)
        rng = np.random.default_rng(pf)
        rf = lf.mask * o.from_global(lf, rng.standard_normal(lf.n_global))
        ec = lc.mask * o.from_global(lc, rng.standard_normal(lc.n_global))
        lhs = o.dot(lc, o.restrict(lf, lc, rf), ec)
        rhs_ = o.dot(lf, rf, o.prolong(lf, lc, ec))
        assert abs(lhs - rhs_) < 1e-12 * max(1.0, abs(lhs))
    # prolongation reproduces a global polynomial of the coarse degree on an affine mesh
    Va = wl.vertex_lattice(nel)
    lf = o.make_level(Va, nel, 5, bc=("N",) * 6, amp=0.0)
    lc = o.make_level(Va, nel, 3, bc=("N",) * 6, amp=0.0)
    poly = lambda X: X[0] ** 3 - 2 * X[1] ** 2 * X[2] + X[0] * X[1] * X[2] + 1
    assert np.allclose(o.prolong(lf, lc, poly(lc.X)), poly(lf.X), atol=1e-12)


@pytest.mark.parametrize("smoother", ["ras", "jacobi"])
def test_vcycle_linear_and_contracting(mg_case, smoother):
    V, nel = mg_case
    pmg = o.pmg_setup(V, nel, (3, 1), smoother=smoother, order=2, coarse_tol=1e-14, coarse_maxit=2000)
    lv = pmg.levels[0]
    rng = np.random.default_rng(3)
    a = lv.mask * o.from_global(lv, rng.standard_normal(lv.n_global))
    b = lv.mask * o.from_global(lv, rng.standard_normal(lv.n_global))
    va, vb, vab = o.vcycle(pmg, a), o.vcycle(pmg, b), o.vcycle(pmg, a + 2 * b)
    assert np.allclose(vab, va + 2 * vb, atol=1e-9 * np.abs(vab).max())
    cols = free_nodes(lv)
    x, w = o.gll(3)
    Af = assembled_stiffness(lv, x, w)[np.ix_(cols, cols)]
    Mm = operator_matrix(lv, lambda r: o.vcycle(pmg, r), cols)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(len(cols)) - Mm @ Af)))
    assert rho < 0.5


@pytest.mark.parametrize("method", ["fpcg", "fgmres"])
@pytest.mark.parametrize("pre", ["jacobi", "ras", "asm"])
def test_solution_matches_direct_solve(mg_case, method, pre):
    V, nel = mg_case
    lv, b = o.problem(V, nel, 5)
    pmg = None if pre == "jacobi" else o.pmg_setup(V, nel, (5, 3, 1), smoother=pre, order=2)
    xsol, it, rel = o.solve(lv, b, pmg, method=method, tol=1e-10)
    assert rel <= 1e-10 and it < 400
    cols = free_nodes(lv)
    xg, wg = o.gll(5)
    Af = assembled_stiffness(lv, xg, wg)[np.ix_(cols, cols)]
    xd = np.linalg.solve(Af, o.to_global(lv, b)[cols])
    assert np.allclose(o.to_global(lv, xsol)[cols], xd, rtol=0, atol=1e-8 * np.abs(xd).max())
    true_res = b - o.ax(lv, xsol)
    assert math.sqrt(o.dot(lv, true_res, true_res)) <= 1e-9 * math.sqrt(o.dot(lv, b, b))


def test_spectral_convergence():
    nel = (2, 2, 2)
    V = wl.vertex_lattice(nel, 0.05, seed=0)
    errs = []
    for p in (2, 4, 6, 8):
        lv, b = o.problem(V, nel, p)
        x, it, rel = o.solve(lv, b, None, tol=1e-13, maxit=5000)
        errs.append(np.max(np.abs(x - wl.u_exact(*lv.X))))
    for a, b_ in zip(errs, errs[1:]):
        assert b_ < a / 8.0
    assert errs[-1] < 5e-5


def test_projection_guess_is_the_a_orthogonal_projection():
    """The projection onto prior solutions (Secs. 3.2 and 4.2): exact for a right-hand side whose
    solution lies in the span; otherwise the error A^-1 b - xbar is A-orthogonal to every prior
    solution (Galerkin condition) and no element of the span is closer in the A-norm."""
    import numpy as np
    import oracle as o
    import workloads as wl
    nel, p = (2, 2, 1), 3
    V = wl.vertex_lattice(nel, 0.05, seed=4)
    lv = o.make_level(V, nel, p)
    def cont(seed):
        return lv.mask * o.from_global(lv, wl.random_lvector(lv.n_global, seed))
    xs = [cont(s) for s in (1, 2, 3)]
    # solution in the span: recovered exactly
    xt = 0.7 * xs[0] - 1.3 * xs[1] + 0.2 * xs[2]
    assert np.max(np.abs(o.projection_guess(lv, xs, o.ax(lv, xt)) - xt)) <= 1e-12 * np.max(np.abs(xt))
    # a dependent set (a repeated direction) defines the same projection
    b = o.ax(lv, cont(9))
    g = o.projection_guess(lv, xs, b)
    g2 = o.projection_guess(lv, xs + [2.0 * xs[1]], b)
    assert np.max(np.abs(g - g2)) <= 1e-10 * np.max(np.abs(g))
    # Galerkin: (x_i, b - A xbar) = 0, and perturbing xbar inside the span raises the A-norm error
    r = b - o.ax(lv, g)
    for x in xs:
        assert abs(o.dot(lv, x, r)) <= 1e-12 * np.sqrt(o.dot(lv, b, b) * o.dot(lv, x, x))
    xstar = cont(9)
    def err(y):
        e = xstar - y
        return o.dot(lv, e, o.ax(lv, e))
    for x in xs:
        assert err(g + 1e-3 * x) > err(g) and err(g - 1e-3 * x) > err(g)
    assert np.array_equal(o.projection_guess(lv, [], b), np.zeros_like(b))


def map_matrix(lin, lout, fn):
    """Matrix of a linear map between continuous L-vectors of two levels, on free global nodes."""
    cin, cout = free_nodes(lin), free_nodes(lout)
    M = np.zeros((len(cout), len(cin)))
    for n, g in enumerate(cin):
        ug = np.zeros(lin.n_global)
        ug[g] = 1.0
        M[:, n] = o.to_global(lout, fn(lin.mask * o.from_global(lin, ug)))[cout]
    return M


@pytest.mark.parametrize("smoother", ["ras", "asm"])
def test_additive_vcycle_is_the_sum_of_subspace_corrections(smoother):
    """Sec. 2.2.2: without Chebyshev acceleration the Schwarz smoothers use an additive V-cycle,
    smoother and coarse correction applied to the same residual with no post-smoothing.  With an
    exact coarse solve its operator is the sum of the level corrections,
    M = S_0 + P_0 (S_1 + P_1 A_c^-1 P_1^T) P_0^T, built here from the dense matrices of each
    step; the multiplicative cycle of Algorithm 1 is a different operator."""
    nel = (3, 2, 2)
    V = wl.vertex_lattice(nel, 0.05, seed=8)
    pmg = o.pmg_setup(V, nel, (3, 2, 1), smoother=smoother, order=2, coarse_tol=1e-14,
                      coarse_maxit=2000, cycle="additive")
    l0, l1, l2 = pmg.levels
    S0 = map_matrix(l0, l0, o.smoother_op(pmg, 0))
    S1 = map_matrix(l1, l1, o.smoother_op(pmg, 1))
    R0 = map_matrix(l0, l1, lambda r: o.restrict(l0, l1, r))
    R1 = map_matrix(l1, l2, lambda r: o.restrict(l1, l2, r))
    P0 = map_matrix(l1, l0, lambda e: o.prolong(l0, l1, e))
    P1 = map_matrix(l2, l1, lambda e: o.prolong(l1, l2, e))
    Ac = map_matrix(l2, l2, lambda u: o.ax(l2, u))
    Mdef = S0 + P0 @ (S1 + P1 @ np.linalg.solve(Ac, R1)) @ R0
    Madd = map_matrix(l0, l0, lambda r: o.vcycle(pmg, r))
    assert np.allclose(Madd, Mdef, rtol=0, atol=1e-10 * np.abs(Mdef).max())
    pmg.cycle = "mult"
    Mmult = map_matrix(l0, l0, lambda r: o.vcycle(pmg, r))
    assert not np.allclose(Mmult, Mdef, rtol=0, atol=1e-3 * np.abs(Mdef).max())


@pytest.mark.parametrize("method", ["fpcg", "fgmres"])
@pytest.mark.parametrize("pre", ["ras", "asm"])
def test_additive_cycle_solution_matches_direct_solve(mg_case, method, pre):
    V, nel = mg_case
    lv, b = o.problem(V, nel, 5)
    pmg = o.pmg_setup(V, nel, (5, 3, 1), smoother=pre, order=0, cycle="additive")
    xsol, it, rel = o.solve(lv, b, pmg, method=method, tol=1e-10)
    assert rel <= 1e-10 and it < 400
    cols = free_nodes(lv)
    xg, wg = o.gll(5)
    Af = assembled_stiffness(lv, xg, wg)[np.ix_(cols, cols)]
    xd = np.linalg.solve(Af, o.to_global(lv, b)[cols])
    assert np.allclose(o.to_global(lv, xsol)[cols], xd, rtol=0, atol=1e-8 * np.abs(xd).max())


def _level_matrices(pmg, l):
    """Dense matrices of level l on its free global nodes: stiffness by brute-force quadrature
    (no sum factorisation), the smoother S, and the transfers to level l+1."""
    lv = pmg.levels[l]
    x, w = o.gll(lv.p)
    cols = free_nodes(lv)
    A = assembled_stiffness(lv, x, w)[np.ix_(cols, cols)]
    if l == len(pmg.levels) - 1:
        return A, None, None, None
    lc = pmg.levels[l + 1]
    S = map_matrix(lv, lv, o.smoother_op(pmg, l))
    R = map_matrix(lv, lc, lambda r: o.restrict(lv, lc, r))
    P = map_matrix(lc, lv, lambda e: o.prolong(lv, lc, e))
    return A, S, R, P


def multiplicative_cycle_matrix(pmg):
    """Algorithm 1 written as an error propagator, from dense matrices only.

    On level l the Chebyshev smoother of Algorithm 2 is the linear map C_l with
    I - C_l A_l = T_{k+1}((theta - S_l A_l)/delta) / T_{k+1}(theta/delta), the polynomial built
    by the three-term recurrence (not by the oracle's Chebyshev routine).  Pre-smoothing, the
    coarse-grid correction with the re-evaluated residual, and post-smoothing give
        I - M_l A_l = (I - C_l A_l) (I - P_l M_{l+1} R_l A_l) (I - C_l A_l),
    with M_coarsest = A_coarsest^-1 (exact coarse solve).  Returns M_0."""
    mats = [_level_matrices(pmg, l) for l in range(len(pmg.levels))]
    M = np.linalg.inv(mats[-1][0])
    for l in range(len(pmg.levels) - 2, -1, -1):
        A, S, R, P = mats[l]
        lmin, lmax = pmg.bounds[l]
        I = np.eye(len(A))
        Esm = chebyshev_matrix_polynomial(S @ A, lmin, lmax, pmg.order[l] + 1)
        Ecg = I - P @ M @ R @ A
        M = (I - Esm @ Ecg @ Esm) @ np.linalg.inv(A)
    return M, mats


@pytest.mark.parametrize("smoother", ["jacobi", "ras", "asm"])
def test_vcycle_is_the_composition_of_algorithm_1(smoother):
    """Algorithm 1 (Sec. 2.2.2) with an exact coarse solve equals the product of its steps'
    error propagators (pre-smoothing, coarse correction, post-smoothing) built from dense
    matrices, on a three-level schedule.  A cycle that drops the post-smoothing, the
    pre-smoothing or the residual re-evaluation is a different operator and fails here."""
    nel = (3, 2, 2)
    V = wl.vertex_lattice(nel, 0.05, seed=8)
    pmg = o.pmg_setup(V, nel, (3, 2, 1), smoother=smoother, order=[2, 1, 0], coarse_tol=1e-14,
                      coarse_maxit=2000)
    l0 = pmg.levels[0]
    Mdef, mats = multiplicative_cycle_matrix(pmg)
    Mv = map_matrix(l0, l0, lambda r: o.vcycle(pmg, r))
    scale = np.abs(Mdef).max()
    assert np.allclose(Mv, Mdef, rtol=0, atol=1e-9 * scale)
    if smoother == "jacobi":
        # S = D^-1 and R = P^T make every step self-adjoint: the cycle is symmetric
        assert np.allclose(Mv, Mv.T, rtol=0, atol=1e-9 * scale)
        A0, S0, R0, P0 = mats[0]
        assert np.allclose(R0, P0.T, rtol=0, atol=1e-13 * np.abs(P0).max())

    # the same composition discriminates the variants of the cycle
    A0, S0, R0, P0 = mats[0]
    lmin, lmax = pmg.bounds[0]

    def cheb(r):
        return o.chebyshev(r, lambda u: o.ax(l0, u), o.smoother_op(pmg, 0), lmin, lmax,
                           pmg.order[0])

    def coarse(r):
        return o.prolong(l0, pmg.levels[1], o.vcycle(pmg, o.restrict(l0, pmg.levels[1], r), 1))

    def no_post(b):
        x = cheb(b)
        return x + coarse(b - o.ax(l0, x))

    def no_pre(b):
        x = coarse(b)
        return x + cheb(b - o.ax(l0, x))

    def stale_residual(b):
        x = cheb(b)
        x = x + coarse(b)
        return x + cheb(b - o.ax(l0, x))

    for variant in (no_post, no_pre, stale_residual):
        Mw = map_matrix(l0, l0, variant)
        assert not np.allclose(Mw, Mdef, rtol=0, atol=1e-4 * scale), variant.__name__


def _textbook_pcg(A, Minv, b, dotf, iters):
    """Preconditioned CG with beta = (z_{k+1}, r_{k+1}) / (z_k, r_k), x0 = 0, fixed count."""
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv(r)
    pv = z.copy()
    rz = dotf(r, z)
    for _ in range(iters):
        w = A(pv)
        alpha = rz / dotf(pv, w)
        x = x + alpha * pv
        r = r - alpha * w
        z = Minv(r)
        rz_new = dotf(r, z)
        pv = z + (rz_new / rz) * pv
        rz = rz_new
    return x


def _fpcg_case():
    nel = (2, 2, 2)
    V = wl.vertex_lattice(nel, 0.1, seed=4)
    lv, b = o.problem(V, nel, 4)
    d = o.jacobi_diag(lv)
    return lv, b, d


def test_fpcg_reduces_to_textbook_pcg_for_a_fixed_preconditioner():
    """With a fixed symmetric positive definite preconditioner (z_{k+1}, r_k) = 0 in exact
    arithmetic, so the flexible beta of Sec. 2.2 equals the textbook one and the iterates of
    the two methods agree step by step."""
    lv, b, d = _fpcg_case()
    A = lambda u: o.ax(lv, u)
    M = lambda r: lv.mask * r / d
    dotf = lambda a, c: o.dot(lv, a, c)
    for k in (1, 2, 5, 12, 20):
        xf, it, _ = o.fpcg(A, M, b, np.zeros_like(b), dotf, tol=0.0, maxit=k)
        assert it == k
        xt = _textbook_pcg(A, M, b, dotf, k)
        assert np.max(np.abs(xf - xt)) <= 1e-12 * np.max(np.abs(xt)), k


def test_fpcg_keeps_consecutive_directions_conjugate_under_a_varying_preconditioner():
    """The flexible beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k) is the one that makes each new
    search direction A-conjugate to the previous one, (p_{k+1}, A p_k) = 0, whatever the
    preconditioner does between iterations (here: a different positive diagonal scaling per
    call).  The search directions are read off the operator's inputs.  The textbook beta loses
    the property under the same preconditioner."""
    lv, b, d = _fpcg_case()
    dotf = lambda a, c: o.dot(lv, a, c)
    rng = np.random.default_rng(11)

    def run(method):
        seen = []

        def A(u):
            seen.append(u.copy())
            return o.ax(lv, u)

        def M(r):
            s = o.from_global(lv, rng.uniform(0.2, 5.0, lv.n_global))
            return lv.mask * r * s / d

        if method == "flexible":
            o.fpcg(A, M, b, np.zeros_like(b), dotf, tol=0.0, maxit=8)
            dirs = seen[1:]                       # the first call forms r_0 = b - A x_0
        else:
            _textbook_pcg(A, M, b, dotf, 8)
            dirs = seen
        cos = []
        for pk, pn in zip(dirs, dirs[1:]):
            Apk = o.ax(lv, pk)
            cos.append(abs(dotf(pn, Apk)) / math.sqrt(dotf(pn, o.ax(lv, pn)) * dotf(pk, Apk)))
        return np.array(cos)

    assert run("flexible").max() <= 1e-12
    assert run("textbook").max() >= 1e-3


def test_fgmres_residual_is_the_krylov_minimum():
    """Right-preconditioned GMRES (Sec. 2.2) with a fixed preconditioner and no restart within k
    steps: its residual after k steps is the smallest of ||r_0 - A M q|| over q in the Krylov space
    span{r_0, (A M) r_0, ..., (A M)^{k-1} r_0} (unique-node 2-norm), computed here from the
    brute-force assembled matrix by a dense least-squares solve.  Errors in the Givens rotations,
    the back substitution or the x update change the residual and fail the comparison."""
    nel = (2, 2, 2)
    V = wl.vertex_lattice(nel, 0.1, seed=4)
    lv, b = o.problem(V, nel, 3)
    d = o.jacobi_diag(lv)
    cols = free_nodes(lv)
    xg, wg = o.gll(3)
    Af = assembled_stiffness(lv, xg, wg)[np.ix_(cols, cols)]
    Mf = np.diag(1.0 / np.diag(Af))
    r0 = o.to_global(lv, b)[cols]
    A = lambda u: o.ax(lv, u)
    M = lambda r: lv.mask * r / d
    dotf = lambda a, c: o.dot(lv, a, c)
    AM = Af @ Mf
    for k in (1, 2, 4, 7):
        x, it, _ = o.fgmres(A, M, b, np.zeros_like(b), dotf, m=20, tol=0.0, maxit=k)
        assert it == k
        res = np.linalg.norm(r0 - Af @ o.to_global(lv, x)[cols])
        K = np.empty((len(cols), k))
        v = r0.copy()
        for j in range(k):
            K[:, j] = v / np.linalg.norm(v)
            v = AM @ K[:, j]
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(AM @ Q, r0, rcond=None)
        best = np.linalg.norm(r0 - AM @ Q @ y)
        assert abs(res - best) <= 1e-9 * np.linalg.norm(r0), (k, res, best)
    # restarted: two cycles of two steps end where two minimisations from the first iterate end
    x2, it2, _ = o.fgmres(A, M, b, np.zeros_like(b), dotf, m=2, tol=0.0, maxit=4)
    r = r0.copy()
    xs = np.zeros(len(cols))
    for _ in range(2):
        K = np.stack([r / np.linalg.norm(r), AM @ r / np.linalg.norm(AM @ r)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(AM @ Q, r, rcond=None)
        xs = xs + Mf @ (Q @ y)
        r = r0 - Af @ xs
    assert np.allclose(o.to_global(lv, x2)[cols], xs, rtol=0, atol=1e-9 * np.abs(xs).max())
