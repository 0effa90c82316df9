"""Brute-force dense matrices used to pin the oracle (CPU only, tiny meshes).

Nothing here uses the oracle's sum factorisation, derivative matrix or geometric factors: the
Lagrange basis and its derivative are built as explicit polynomials (numpy.polynomial), the
Jacobian of the isoparametric map is formed point by point from those polynomials, and the
element stiffness A^e_IJ = sum_q w_q |det J| (J^-T grad phi_I).(J^-T grad phi_J) (Sec. 2.1) is
assembled entry by entry into the global matrix.
"""
import numpy as np
from numpy.polynomial import polynomial as P


def lagrange_polys(nodes):
    """Coefficient arrays of h_j and h_j' (power basis) for the given nodes."""
    n = len(nodes)
    hs, dhs = [], []
    for j in range(n):
        c = np.array([1.0])
        for m in range(n):
            if m != j:
                c = P.polymul(c, np.array([-nodes[m], 1.0]) / (nodes[j] - nodes[m]))
        hs.append(c)
        dhs.append(P.polyder(c))
    return hs, dhs


def element_stiffness(Xe, nodes, weights):
    """Dense (N^3 x N^3) stiffness of one element with node coordinates Xe[c, k, j, i]."""
    N = len(nodes)
    hs, dhs = lagrange_polys(nodes)
    Hv = np.array([[P.polyval(x, h) for x in nodes] for h in hs])      # Hv[j, q] = h_j(xi_q)
    dHv = np.array([[P.polyval(x, h) for x in nodes] for h in dhs])    # dHv[j, q] = h_j'(xi_q)
    nb = N ** 3
    Ae = np.zeros((nb, nb))
    basis = [(i, j, k) for k in range(N) for j in range(N) for i in range(N)]
    for qc in range(N):
        for qb in range(N):
            for qa in range(N):
                # reference gradients of every basis function at q = (qa, qb, qc)
                gr = np.array([[dHv[i, qa] * Hv[j, qb] * Hv[k, qc],
                                Hv[i, qa] * dHv[j, qb] * Hv[k, qc],
                                Hv[i, qa] * Hv[j, qb] * dHv[k, qc]] for (i, j, k) in basis])
                # Jacobian dx_c/dr_a at q from the map x = sum x_ijk phi_ijk
                Jm = np.zeros((3, 3))
                for n_, (i, j, k) in enumerate(basis):
                    Jm += np.outer(Xe[:, k, j, i], gr[n_])
                detJ = np.linalg.det(Jm)
                gphys = gr @ np.linalg.inv(Jm)          # rows: grad phi in physical coords
                wq = weights[qa] * weights[qb] * weights[qc]
                Ae += wq * abs(detJ) * gphys @ gphys.T
    return Ae


def assembled_stiffness(lv, nodes, weights):
    """Global stiffness Q^T A_L Q (all global nodes, no mask)."""
    n = lv.n_global
    A = np.zeros((n, n))
    N = lv.p + 1
    for e in range(lv.E):
        Ae = element_stiffness(lv.X[:, e], nodes, weights)
        g = lv.gid[e].reshape(-1)                   # ordered k, j, i with i fastest
        A[np.ix_(g, g)] += Ae
    return A


def free_nodes(lv):
    """Sorted global ids of the nodes not on a Dirichlet face."""
    fm = np.zeros(lv.n_global, dtype=bool)
    fm[lv.gid[lv.mask > 0]] = True
    return np.nonzero(fm)[0]
