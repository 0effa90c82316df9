"""The skewed lattice (a stand-in for the paper's Kershaw meshes, Sec. 3.1) and the oracle's
geometry on its sheared, high-aspect-ratio elements.

Pins: eps = 1 is the uniform box; the boundary stays on the unit cube; every column of
vertices is strictly increasing, with width ratios (2 - eps)/eps; and, since each coordinate
function is in the isoparametric space and det J of a trilinear map is integrated exactly by
GLL quadrature at p >= 2, the discrete energies of the coordinate functions are exactly those of
the continuum: (x_i, A x_j) = delta_ij |Omega| = delta_ij with Neumann conditions, A 1 = 0 and
sum B = 1.  A wrong or transposed off-diagonal geometric factor (the sheared elements have
large G_rs, G_rt, G_st) breaks the cross energies.
"""
import numpy as np
import pytest

import oracle as o
import workloads as wl


def test_lattice_shape_and_limits():
    nel = (6, 4, 5)
    assert np.array_equal(wl.skewed_lattice(nel, 1.0), wl.vertex_lattice(nel))
    for eps in (0.3, 0.05):
        V = wl.skewed_lattice((12, 12, 12), eps, segments=6)
        assert np.allclose(V[..., 0, 0], 0) and np.allclose(V[..., -1, 0], 1)
        assert np.allclose(V[:, 0, :, 1], 0) and np.allclose(V[:, -1, :, 1], 1)
        assert np.allclose(V[0, :, :, 2], 0) and np.allclose(V[-1, :, :, 2], 1)
        dy = np.diff(V[..., 1], axis=1)
        dz = np.diff(V[..., 2], axis=0)
        assert dy.min() > 0 and dz.min() > 0
        assert dy.max() / dy.min() == pytest.approx((2 - eps) / eps)
        assert dz.max() / dz.min() == pytest.approx((2 - eps) / eps)


@pytest.mark.parametrize("eps", [0.3, 0.05])
def test_coordinate_energies_are_exact(eps):
    nel, p = (4, 4, 4), 3     # the zigzag takes 1, 0, -1, 0, 1 at the vertex planes: sheared
    lv = o.make_level(wl.skewed_lattice(nel, eps), nel, p, bc=("N",) * 6, amp=0.0)
    assert lv.detJ.min() > 0
    assert float(lv.B.sum()) == pytest.approx(1.0, abs=1e-13)
    ones = np.ones(lv.gid.shape)
    assert np.max(np.abs(o.ax(lv, ones, mask=False))) <= 1e-12
    X = [lv.X[i] for i in range(3)]
    E = np.array([[o.dot(lv, X[i], o.ax(lv, X[j], mask=False)) for j in range(3)] for i in range(3)])
    assert np.max(np.abs(E - np.eye(3))) <= 1e-12, E
    # the elements really are sheared: the off-diagonal factors do not vanish
    assert np.max(np.abs(lv.G[1])) > 0.1 * np.max(np.abs(lv.G[0]))
