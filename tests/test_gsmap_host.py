"""Host logic of the index-map QQ^T (Sec. 2.1): the local copies of each global node grouped by
global id and bucketed by multiplicity (se_gsmap_count runs the same grouping se_gsmap_create
uploads, with no device call).

Pins: on a box lattice of nx x ny x nz elements of order p, the multiplicity of a global node is
the number of elements around it, so the bucket sizes have closed forms (faces, edges and
vertices of the element lattice, inside the box or on its boundary); relabelling the global ids
(sparse labels take the sorting path instead of the counting sort) changes nothing; random
connectivities are checked against a histogram of the ids.
"""
import numpy as np
import pytest

import oracle as o
import workloads as wl
from paper_2110_07663_gb300 import se


def box_counts(nx, ny, nz, p):
    """(pairs, quads, octets, other, masked singles) of an all-Dirichlet box lattice."""
    q = p - 1  # nodes strictly inside an element edge
    # 8 copies: lattice vertices inside the box
    n8 = (nx - 1) * (ny - 1) * (nz - 1)
    # 4 copies: interior element edges (inside the box), lattice vertices inside a box face
    n4 = q * (nx * (ny - 1) * (nz - 1) + ny * (nx - 1) * (nz - 1) + nz * (nx - 1) * (ny - 1))
    n4 += 2 * ((nx - 1) * (ny - 1) + (nx - 1) * (nz - 1) + (ny - 1) * (nz - 1))
    # 2 copies: interior element faces, element edges inside a box face, lattice vertices inside
    # a box edge
    n2 = q * q * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))
    n2 += 2 * q * (nx * (ny - 1) + ny * (nx - 1) + nx * (nz - 1) + nz * (nx - 1)
                   + ny * (nz - 1) + nz * (ny - 1))
    n2 += 4 * ((nx - 1) + (ny - 1) + (nz - 1))
    # 1 copy on the boundary (all Dirichlet): boundary element faces, box edges, box corners
    n1 = q * q * 2 * (nx * ny + ny * nz + nx * nz) + q * 4 * (nx + ny + nz) + 8
    return (n2, n4, n8, 0, n1)


def histogram_counts(gid, dirichlet):
    uniq, inv, cnt = np.unique(np.asarray(gid).ravel(), return_inverse=True, return_counts=True)
    masked = np.zeros(len(uniq), dtype=bool)
    if dirichlet is not None:
        np.logical_or.at(masked, inv.ravel(), np.asarray(dirichlet).ravel() != 0)
    other = (cnt >= 2) & (cnt != 2) & (cnt != 4) & (cnt != 8)
    return (int(np.sum(cnt == 2)), int(np.sum(cnt == 4)), int(np.sum(cnt == 8)),
            int(np.sum(other)), int(np.sum((cnt == 1) & masked)))


@pytest.mark.parametrize("nel,p", [((1, 1, 1), 2), ((2, 2, 2), 1), ((3, 2, 4), 3), ((4, 4, 4), 7),
                                   ((2, 3, 1), 5)])
def test_box_lattice_counts_closed_form(nel, p):
    lv = o.make_level(wl.vertex_lattice(nel, 0.0, 0), nel, p)
    dirichlet = (lv.mask == 0).astype(np.uint8)
    got = se.se_gsmap_count(lv.gid, dirichlet)
    assert got == box_counts(*nel, p)
    # the same map with every global id relabelled sparsely (sorting path)
    assert se.se_gsmap_count(lv.gid * 1000003 + 10 ** 12, dirichlet) == got
    # without a mask no single copy is kept
    assert se.se_gsmap_count(lv.gid)[:4] == got[:4] and se.se_gsmap_count(lv.gid)[4] == 0


def test_mixed_boundary_counts():
    nel, p = (3, 2, 2), 4
    bc = ("N", "D", "N", "N", "D", "N")
    lv = o.make_level(wl.vertex_lattice(nel, 0.05, 1), nel, p, bc)
    dirichlet = (lv.mask == 0).astype(np.uint8)
    assert se.se_gsmap_count(lv.gid, dirichlet) == histogram_counts(lv.gid, dirichlet)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_connectivity_counts(seed):
    rng = np.random.default_rng(seed)
    mult = rng.integers(1, 10, size=400)             # multiplicities 1..9
    gid = np.repeat(np.arange(400), mult)
    rng.shuffle(gid)
    dirichlet = (rng.random(gid.size) < 0.05).astype(np.uint8)
    assert se.se_gsmap_count(gid, dirichlet) == histogram_counts(gid, dirichlet)
    assert se.se_gsmap_count(gid * 7919 + 3 * 10 ** 11, dirichlet) == histogram_counts(gid, dirichlet)


def test_invalid_arguments():
    with pytest.raises(se.SeError) as e:
        se.se_gsmap_count(np.array([0, 1, -1, 2]))
    assert e.value.code == se.SE_EINVAL
    with pytest.raises(se.SeError) as e:
        se.se_gsmap_count(np.zeros(0, dtype=np.int64))
    assert e.value.code == se.SE_EINVAL
    with pytest.raises(se.SeError) as e:  # rejected before any device work
        se.se_gsmap_create(np.array([3, -5]))
    assert e.value.code == se.SE_EINVAL
