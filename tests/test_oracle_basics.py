"""Pins of the oracle's 1D building blocks, geometry and operator (CPU only).

Each check is fixed by the mathematics, not by the oracle itself: closed-form GLL rules,
polynomial exactness, brute-force quadrature of the weak form (Sec. 2.1), symmetry, the
constant null space under Neumann conditions, and the surface-node count of Sec. 4.1.
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.dense_reference import assembled_stiffness, free_nodes


# ---------------------------------------------------------------- GLL rules and matrices
@pytest.mark.parametrize("p,nodes,weights", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_gll_closed_forms(p, nodes, weights):
    x, w = o.gll(p)
    assert np.allclose(x, nodes, atol=1e-15, rtol=0)
    assert np.allclose(w, weights, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", range(1, 12))
def test_gll_quadrature_exactness(p):
    x, w = o.gll(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * p):              # exact up to degree 2p-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    # degree 2p is not integrated exactly by a (p+1)-point Lobatto rule
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-9


@pytest.mark.parametrize("p", range(1, 12))
def test_derivative_matrix(p):
    x, _ = o.gll(p)
    D = o.deriv_matrix(x)
    for k in range(p + 1):                  # exact on degree <= p
        d_exact = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        assert np.allclose(D @ x ** k, d_exact, atol=2e-12 * max(1, p * p))
    assert abs(D[0, 0] + p * (p + 1) / 4.0) < 1e-11 * p * p
    assert abs(D[p, p] - p * (p + 1) / 4.0) < 1e-11 * p * p
    # GLL: interior diagonal entries vanish; centro-antisymmetry D_{p-i,p-j} = -D_ij
    assert np.allclose(np.diag(D)[1:-1], 0.0, atol=1e-11 * p * p)
    assert np.allclose(D[::-1, ::-1], -D, atol=1e-11 * p * p)


@pytest.mark.parametrize("pf,pc", [(7, 5), (7, 3), (5, 3), (3, 1), (9, 5), (5, 1), (9, 7)])
def test_interp_reproduces_coarse_polynomials(pf, pc):
    J = o.interp_1d(pf, pc)
    xf, _ = o.gll(pf)
    xc, _ = o.gll(pc)
    for k in range(pc + 1):
        assert np.allclose(J @ xc ** k, xf ** k, atol=1e-13)


# ---------------------------------------------------------------- geometry
def test_affine_box_geometric_factors():
    nel = (3, 2, 2)
    V = wl.vertex_lattice(nel)
    V[..., 0] *= 2.0                         # box [0,2] x [0,1] x [0,1]
    lv = o.make_level(V, nel, 4, amp=0.0)
    hx, hy, hz = 2.0 / 3, 0.5, 0.5
    w = lv.w
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    det = hx * hy * hz / 8.0
    assert np.allclose(lv.G[0], W3 * det * (2 / hx) ** 2)
    assert np.allclose(lv.G[3], W3 * det * (2 / hy) ** 2)
    assert np.allclose(lv.G[5], W3 * det * (2 / hz) ** 2)
    for c in (1, 2, 4):
        assert np.allclose(lv.G[c], 0.0, atol=1e-14)
    assert abs(lv.B.sum() - 2.0) < 1e-13


def test_mapped_box_volume_and_jacobian():
    # the smooth map fixes the boundary, so the mapped domain is the unit cube
    V = wl.vertex_lattice((4, 4, 4), 0.05, seed=3)
    lv = o.make_level(V, (4, 4, 4), 7, amp=0.05)
    assert lv.detJ.min() > 0
    assert abs(lv.B.sum() - 1.0) < 1e-6
    # node coordinates follow the stated map at a corner node
    x0 = V[0, 0, 0]
    assert np.allclose(lv.X[:, 0, 0, 0, 0], x0 + 0.05 * np.prod(np.sin(2 * np.pi * x0)))


# ---------------------------------------------------------------- operator vs brute force
def dense_from_oracle(lv, mask=True):
    """Columns of the oracle's assembled operator on free (or all) global nodes."""
    cols = free_nodes(lv) if mask else np.arange(lv.n_global)
    A = np.zeros((len(cols), len(cols)))
    for n, g in enumerate(cols):
        ug = np.zeros(lv.n_global)
        ug[g] = 1.0
        y = o.ax(lv, o.from_global(lv, ug), mask=mask)
        A[:, n] = o.to_global(lv, y)[cols]
    return A, cols


@pytest.mark.parametrize("nel,p,pert,amp", [((2, 2, 2), 2, 0.1, 0.05), ((2, 1, 2), 3, 0.1, 0.05),
                                            ((1, 2, 1), 4, 0.0, 0.05)])
def test_operator_equals_brute_force_quadrature(nel, p, pert, amp):
    V = wl.vertex_lattice(nel, pert, seed=5)
    lv = o.make_level(V, nel, p, amp=amp)
    x, w = o.gll(p)
    Ad = assembled_stiffness(lv, x, w)
    Ao, cols = dense_from_oracle(lv)
    ref = Ad[np.ix_(cols, cols)]
    assert np.max(np.abs(Ao - ref)) <= 1e-13 * np.max(np.abs(ref)) * 10
    An, cols_all = dense_from_oracle(lv, mask=False)
    assert np.max(np.abs(An - Ad)) <= 1e-12 * np.max(np.abs(Ad))


def test_operator_symmetric_psd_and_neumann_nullspace():
    nel = (2, 2, 2)
    V = wl.vertex_lattice(nel, 0.1, seed=1)
    lv = o.make_level(V, nel, 3, bc=("N",) * 6)
    A, _ = dense_from_oracle(lv, mask=False)
    assert np.allclose(A, A.T, atol=1e-13 * np.abs(A).max())
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-12 * ev.max()
    ones = np.ones(lv.gid.shape)
    assert np.max(np.abs(o.ax(lv, ones, mask=False))) < 1e-12
    # Dirichlet on all faces: positive definite
    lvd = o.make_level(V, nel, 3)
    Ad, _ = dense_from_oracle(lvd)
    assert np.linalg.eigvalsh(0.5 * (Ad + Ad.T)).min() > 0


def test_energy_of_polynomial_is_exact_on_affine_mesh():
    nel = (2, 3, 2)
    V = wl.vertex_lattice(nel)
    lv = o.make_level(V, nel, 4, bc=("N",) * 6, amp=0.0)
    X, Y, Z = lv.X
    u = X * X + 2 * X * Y - Z ** 3 + Y
    # integral over [0,1]^3 of |grad u|^2, grad u = (2x+2y, 2x+1, -3z^2)
    exact = (4 / 3 + 2 * 4 / 4 + 4 / 3) + (4 / 3 + 2 + 1) + 9 / 5
    assert abs(o.dot(lv, u, o.ax(lv, u, mask=False)) - exact) < 1e-12


def test_jacobi_diag_equals_assembled_diagonal():
    nel = (2, 2, 1)
    V = wl.vertex_lattice(nel, 0.1, seed=2)
    lv = o.make_level(V, nel, 3, amp=0.05)
    x, w = o.gll(3)
    Ad = assembled_stiffness(lv, x, w)
    d = o.to_global(lv, o.jacobi_diag(lv))
    cols = free_nodes(lv)
    assert np.allclose(d[cols], np.diag(Ad)[cols], rtol=1e-13, atol=0)


@pytest.mark.parametrize("p,shared", [(7, 296), (3, 56), (5, 152), (9, 488)])
def test_surface_node_count(p, shared):
    # Sec. 4.1: 296 of the 512 nodes of a p=7 element lie on its surface, (p+1)^3-(p-1)^3
    nel = (3, 3, 3)
    lv = o.make_level(wl.vertex_lattice(nel), nel, p, bc=("N",) * 6)
    centre = 13
    assert int(np.sum(lv.mult[centre] > 1)) == shared == (p + 1) ** 3 - (p - 1) ** 3
    assert np.allclose(o.qqt(lv, 1.0 / lv.mult), 1.0)       # partition of unity


def test_rhs_and_counter_generator():
    # SplitMix64 published test vector: seed 1234567, first outputs (Vigna's splitmix64.c)
    z = wl.splitmix64(1234567, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in z] == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    u = wl.uniform01(7, np.arange(1000, dtype=np.uint64))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.05
