"""FP64 CPU oracle (numpy): plain, slow, obviously correct.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may use it.

Notation follows the paper (Sec. 2): E elements, polynomial order p, N = p+1 GLL points per
direction, pbar = p+3 points per direction of an extended Schwarz subdomain.  A local vector
(L-vector, u_L = Q u) is an array of shape (E, N, N, N) indexed [e, k, j, i] (i, the r index,
fastest), which flattens to idx = i + N(j + N(k + N e)).  Element e = ex + nx(ey + ny ez) of a
box lattice of nx*ny*nz hexahedra.

Readings of points where the paper is silent are marked READING at the code that takes them.
Parity unpinned against printed results: the paper prints none for these meshes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# =============================================================================================
# 1D building blocks (Sec. 2.1): GLL points and weights, Lagrange cardinal basis h_j,
# derivative matrix D_ij = h_j'(xi_i), interpolation matrices.
# =============================================================================================


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative from (1-x^2) P_n' = n (P_{n-1} - x P_n); valid for |x| < 1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.abs(x) == 1.0
    dp = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gll(p: int):
    """Gauss-Lobatto-Legendre nodes (ascending) and weights on [-1,1] (Sec. 2.1).

    Nodes: -1, +1 and the p-1 roots of P_p'; Newton's method from the Chebyshev-Gauss-Lobatto
    points, using P_p'' from Legendre's equation.  Weights: w_j = 2 / (p(p+1) P_p(xi_j)^2).
    """
    if p < 1:
        raise ValueError("p >= 1")
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    x[0], x[-1] = -1.0, 1.0
    inner = x[1:-1].copy()
    for _ in range(100):
        P, dP = legendre(p, inner)
        d2P = (2.0 * inner * dP - p * (p + 1) * P) / (1.0 - inner * inner)
        dx = dP / d2P
        inner -= dx
        if np.max(np.abs(dx), initial=0.0) < 1e-16:
            break
    x[1:-1] = inner
    if p % 2 == 0:
        x[p // 2] = 0.0
    P, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * P * P)
    return x, w


def lagrange_eval(nodes, x):
    """Matrix J_ij = h_j(x_i) of the Lagrange cardinal basis on ``nodes`` (product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    J = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                J[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return J


def deriv_matrix(nodes):
    """D_ij = h_j'(xi_i) (Sec. 2.1) from the barycentric weights lam_j = 1/prod_{m!=j}(xi_j-xi_m):
    D_ij = (lam_j/lam_i)/(xi_i - xi_j) for i != j, and rows summing to zero."""
    xi = np.asarray(nodes, dtype=np.float64)
    n = len(xi)
    lam = np.array([1.0 / np.prod([xi[j] - xi[m] for m in range(n) if m != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])
        D[i, i] = -np.sum(D[i, :])
    return D


# Tensor contractions along one reference direction of arrays [..., k, j, i].
def along_r(A, u):
    """y[..., k, j, a] = sum_i A[a, i] u[..., k, j, i]."""
    return u @ A.T


def along_s(A, u):
    """y[..., k, b, i] = sum_j A[b, j] u[..., k, j, i]."""
    return np.einsum("bj,...kji->...kbi", A, u)


def along_t(A, u):
    """y[..., c, j, i] = sum_k A[c, k] u[..., k, j, i]."""
    return np.einsum("ck,...kji->...cji", A, u)


# =============================================================================================
# Mesh, isoparametric geometry (Sec. 2.1) and the Boolean gather Q.
# =============================================================================================


@dataclass
class Level:
    """One discretisation level of the box mesh (order p)."""
    nel: tuple
    p: int
    bc: tuple                 # 6 faces (x-, x+, y-, y+, z-, z+): 'D' Dirichlet or 'N' Neumann
    xi: np.ndarray = None
    w: np.ndarray = None
    D: np.ndarray = None
    X: np.ndarray = None      # node coordinates (3, E, N, N, N)
    G: np.ndarray = None      # geometric factors (6, E, N, N, N): rr, rs, rt, ss, st, tt
    B: np.ndarray = None      # diagonal local mass w_i w_j w_k det J
    detJ: np.ndarray = None
    gid: np.ndarray = None    # global node id of each local node (E, N, N, N)
    n_global: int = 0
    mask: np.ndarray = None   # 1.0 where the node is free, 0.0 on Dirichlet faces
    mult: np.ndarray = None   # number of local copies of the node
    lattice: tuple = None     # global node lattice extents (NX, NY, NZ)
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.p + 1

    @property
    def E(self):
        return self.nel[0] * self.nel[1] * self.nel[2]


def element_corners(V, nel):
    """Corner vertices of every element: array (E, 2, 2, 2, 3) indexed [e, dz, dy, dx, c]."""
    nx, ny, nz = nel
    C = np.empty((nz, ny, nx, 2, 2, 2, 3))
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                C[:, :, :, dz, dy, dx, :] = V[dz:dz + nz, dy:dy + ny, dx:dx + nx, :]
    return C.reshape(nx * ny * nz, 2, 2, 2, 3)


def node_coordinates(V, nel, p, amp):
    """GLL node positions x_ijk^e of the mapped box (Sec. 2.1, isoparametric map).

    Trilinear map of each element's 8 lattice vertices to its GLL points, then the smooth map
    x_c <- x_c + amp sin(2 pi x) sin(2 pi y) sin(2 pi z) for every coordinate c, evaluated at the
    trilinear position.  READING: the same scalar is added to x, y and z.
    """
    xi, _ = gll(p)
    C = element_corners(V, nel)
    phi = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0])   # phi[d, i]
    # x[e, k, j, i, c] = sum_{dz,dy,dx} C[e,dz,dy,dx,c] phi[dz,k] phi[dy,j] phi[dx,i]
    x = np.einsum("ezyxc,zk,yj,xi->ekjic", C, phi, phi, phi)
    s = np.sin(2 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1]) * np.sin(2 * np.pi * x[..., 2])
    x = x + amp * s[..., None]
    return np.moveaxis(x, -1, 0).copy()


def geometric_factors(X, D, w):
    """G_ab = w_i w_j w_k det(J) (grad r_a . grad r_b) and B = w_i w_j w_k det(J) (Sec. 2.1).

    J_ca = dx_c/dr_a from the derivative matrix applied to the node coordinates.
    """
    Jm = np.empty(X.shape[1:] + (3, 3))
    for c in range(3):
        Jm[..., c, 0] = along_r(D, X[c])
        Jm[..., c, 1] = along_s(D, X[c])
        Jm[..., c, 2] = along_t(D, X[c])
    detJ = np.linalg.det(Jm)
    Jinv = np.linalg.inv(Jm)                           # Jinv[..., a, c] = dr_a/dx_c
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    scale = W3[None] * detJ
    idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    G = np.stack([scale * np.sum(Jinv[..., a, :] * Jinv[..., b, :], axis=-1) for a, b in idx])
    return G, scale, detJ


def lattice_indices(nel, p):
    """Global lattice coordinates (I, J, K) of every local node: I = ex p + i, etc."""
    nx, ny, nz = nel
    N = p + 1
    e = np.arange(nx * ny * nz)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    r = np.arange(N)
    I = ex[:, None, None, None] * p + r[None, None, None, :]
    J = ey[:, None, None, None] * p + r[None, None, :, None]
    K = ez[:, None, None, None] * p + r[None, :, None, None]
    shape = (len(e), N, N, N)
    return np.broadcast_to(I, shape), np.broadcast_to(J, shape), np.broadcast_to(K, shape)


def make_level(V, nel, p, bc=("D",) * 6, amp=0.05):
    """Build a level: geometry, Q (global ids), Dirichlet mask, multiplicity (Sec. 2.1)."""
    lv = Level(nel=tuple(nel), p=p, bc=tuple(bc))
    lv.xi, lv.w = gll(p)
    lv.D = deriv_matrix(lv.xi)
    lv.X = node_coordinates(V, nel, p, amp)
    lv.G, lv.B, lv.detJ = geometric_factors(lv.X, lv.D, lv.w)
    nx, ny, nz = nel
    NX, NY, NZ = nx * p + 1, ny * p + 1, nz * p + 1
    lv.lattice = (NX, NY, NZ)
    I, J, K = lattice_indices(nel, p)
    lv.gid = (I + NX * (J + NY * K)).astype(np.int64)
    lv.n_global = NX * NY * NZ
    free = np.ones(lv.gid.shape, dtype=bool)
    for face, (arr, lim) in enumerate([(I, 0), (I, NX - 1), (J, 0), (J, NY - 1), (K, 0), (K, NZ - 1)]):
        if bc[face] == "D":
            free &= arr != lim
    lv.mask = free.astype(np.float64)
    counts = np.bincount(lv.gid.ravel(), minlength=lv.n_global)
    lv.mult = counts[lv.gid].astype(np.float64)
    return lv


# =============================================================================================
# Operator (Sec. 2.1): A = Q^T A_L Q, masked; QQ^T direct stiffness summation.
# =============================================================================================


def qqt(lv, u):
    """QQ^T u: every local copy of a global node receives the sum over all copies."""
    s = np.bincount(lv.gid.ravel(), weights=u.ravel(), minlength=lv.n_global)
    return s[lv.gid]


def to_global(lv, u):
    """Global vector of a continuous L-vector (Q^+ u): the value held by the copies."""
    s = np.bincount(lv.gid.ravel(), weights=(u / lv.mult).ravel(), minlength=lv.n_global)
    return s


def from_global(lv, ug):
    """Q u: scatter a global vector to all local copies."""
    return ug[lv.gid]


def ax_local(lv, u):
    """A_L u, element by element: y = sum_a D_a^T (sum_b G_ab D_b u) (Sec. 2.1, tensor-product
    sum factorisation; 12E(p+1)^4 operations, Sec. 1)."""
    D = lv.D
    ur, us, ut = along_r(D, u), along_s(D, u), along_t(D, u)
    Grr, Grs, Grt, Gss, Gst, Gtt = lv.G
    wr = Grr * ur + Grs * us + Grt * ut
    ws = Grs * ur + Gss * us + Gst * ut
    wt = Grt * ur + Gst * us + Gtt * ut
    return along_r(D.T, wr) + along_s(D.T, ws) + along_t(D.T, wt)


def ax(lv, u, mask=True):
    """Assembled operator on continuous L-vectors: y = M QQ^T A_L M u (Sec. 2.1).
    READING: the Dirichlet space X_0 is imposed by masking the input and the output."""
    if mask:
        return lv.mask * qqt(lv, ax_local(lv, lv.mask * u))
    return qqt(lv, ax_local(lv, u))


def dot(lv, a, b):
    """Inner product of two continuous L-vectors counting each global node once."""
    return float(np.sum(a * b / lv.mult))


def rhs(lv, f_nodes):
    """b = M QQ^T (B_L f) with the diagonal GLL mass matrix (Sec. 2.1, eq. 3)."""
    return lv.mask * qqt(lv, lv.B * f_nodes)


def jacobi_diag(lv):
    """diag(A) = QQ^T diag(A_L) (Sec. 2.2.3, Jacobi surrogate), element diagonal in closed form:
    sum_l D_li^2 G_rr(l,j,k) + ... + 2 D_ii D_jj G_rs(i,j,k) + 2 D_ii D_kk G_rt + 2 D_jj D_kk G_st."""
    D = lv.D
    D2 = D * D
    Grr, Grs, Grt, Gss, Gst, Gtt = lv.G
    d = along_r(D2.T, Grr) + along_s(D2.T, Gss) + along_t(D2.T, Gtt)
    dd = np.diag(D)
    di = dd[None, None, None, :]
    dj = dd[None, None, :, None]
    dk = dd[None, :, None, None]
    d = d + 2.0 * (di * dj * Grs + di * dk * Grt + dj * dk * Gst)
    dg = qqt(lv, d)
    return np.where(lv.mask > 0, dg, 1.0)


# =============================================================================================
# Overlapping Schwarz smoother with fast-diagonalisation local solves (Sec. 2.2.2, eqs 4-9).
# =============================================================================================


def element_box_lengths(V, nel, amp=0.05):
    """Box-like approximation of each deformed element (Sec. 2.2.2, Fig. 1a).

    READING: length along direction d = mean of the 4 corner-to-corner edge lengths of the mapped
    element along d (corners after the smooth map).  Returns array (E, 3).
    """
    C = element_corners(V, nel).copy()              # [e, dz, dy, dx, c]
    s = np.sin(2 * np.pi * C[..., 0]) * np.sin(2 * np.pi * C[..., 1]) * np.sin(2 * np.pi * C[..., 2])
    C = C + amp * s[..., None]
    lx = np.linalg.norm(C[:, :, :, 1, :] - C[:, :, :, 0, :], axis=-1).mean(axis=(1, 2))
    ly = np.linalg.norm(C[:, :, 1, :, :] - C[:, :, 0, :, :], axis=-1).mean(axis=(1, 2))
    lz = np.linalg.norm(C[:, 1, :, :, :] - C[:, 0, :, :, :], axis=-1).mean(axis=(1, 2))
    return np.stack([lx, ly, lz], axis=1)


def fdm_1d(p, lengths, has_left, has_right, dir_left, dir_right):
    """Extended 1D stiffness/mass pairs (A_*, B_*) of element directions (Sec. 2.2.2).

    For each row of ``lengths`` = (l_left, l, l_right), the 1D GLL stiffness (2/l) D^T W D and
    mass (l/2) W are assembled over the left neighbour, the element and the right neighbour; the
    extended window keeps pbar = p+3 points: left neighbour node p-1, own nodes 0..p, right
    neighbour node 1 (Fig. 1b); beyond the window the local problem is homogeneous Dirichlet.
    READING: a side without a neighbour drops its extension point, and on a Dirichlet side also
    the own boundary node.  Returns (Abar (M,n,n), Bbar diagonal (M,n), active) with ``active``
    the kept window positions (0..p+2), the same for all rows.
    """
    lengths = np.atleast_2d(np.asarray(lengths, dtype=np.float64))
    xi, w = gll(p)
    D = deriv_matrix(xi)
    N = p + 1
    Ke = D.T @ np.diag(w) @ D
    M = lengths.shape[0]
    n1 = 3 * p + 1
    A1 = np.zeros((M, n1, n1))
    B1 = np.zeros((M, n1))
    for s in range(3):
        if (s == 0 and not has_left) or (s == 2 and not has_right):
            continue                      # no neighbour: no segment beyond this side
        o = s * p
        l = lengths[:, s]
        A1[:, o:o + N, o:o + N] += (2.0 / l)[:, None, None] * Ke[None]
        B1[:, o:o + N] += (l / 2.0)[:, None] * w[None]
    window = [p - 1] + [p + i for i in range(N)] + [2 * p + 1]     # positions 0..p+2
    active = []
    for pos in range(p + 3):
        if pos == 0 and not has_left:
            continue
        if pos == p + 2 and not has_right:
            continue
        if pos == 1 and (not has_left) and dir_left:
            continue
        if pos == p + 1 and (not has_right) and dir_right:
            continue
        active.append(pos)
    idx = np.array([window[q] for q in active])
    return A1[:, idx[:, None], idx[None, :]], B1[:, idx], active


def fdm_factors(p, lengths, has_left, has_right, dir_left, dir_right):
    """S_* and Lambda_* of eqs 6-7: A s = lam B s with S^T A S = Lambda, S^T B S = I.

    Solved through the symmetric matrix B^-1/2 A B^-1/2 = V Lambda V^T, S = B^-1/2 V.  Window
    positions that are not active get zero rows of S; the unused columns are zero with lam = 1.
    Returns S (M, pbar, pbar) and Lambda (M, pbar) for the M rows of ``lengths``.
    """
    pb = p + 3
    Ab, Bd, active = fdm_1d(p, lengths, has_left, has_right, dir_left, dir_right)
    bi = 1.0 / np.sqrt(Bd)
    lam, Vv = np.linalg.eigh(bi[:, :, None] * Ab * bi[:, None, :])
    M, na = Bd.shape
    S = np.zeros((M, pb, pb))
    L = np.ones((M, pb))
    S[:, np.array(active), :na] = bi[:, :, None] * Vv
    L[:, :na] = lam
    return S, L


def fdm_setup(lv, V, amp=0.05):
    """Per element and direction: S (E, 3, pbar, pbar) and Lambda (E, 3, pbar) (eqs 6-7).
    The neighbour lengths are the box lengths of the face neighbours along that direction."""
    nx, ny, nz = lv.nel
    p = lv.p
    pb = p + 3
    lens = element_box_lengths(V, lv.nel, amp)
    E = lv.E
    S = np.zeros((E, 3, pb, pb))
    Lm = np.zeros((E, 3, pb))
    e = np.arange(E)
    ec = np.stack([e % nx, (e // nx) % ny, e // (nx * ny)], axis=1)
    dims = (nx, ny, nz)
    for d in range(3):
        stride = (1, nx, nx * ny)[d]
        hl_all = ec[:, d] > 0
        hr_all = ec[:, d] < dims[d] - 1
        ll = np.where(hl_all, lens[np.maximum(e - stride, 0), d], lens[:, d])
        lr = np.where(hr_all, lens[np.minimum(e + stride, E - 1), d], lens[:, d])
        for hl in (False, True):
            for hr in (False, True):
                sel = np.nonzero((hl_all == hl) & (hr_all == hr))[0]
                if len(sel) == 0:
                    continue
                trip = np.stack([ll[sel], lens[sel, d], lr[sel]], axis=1)
                S[sel, d], Lm[sel, d] = fdm_factors(p, trip, hl, hr,
                                                    lv.bc[2 * d] == "D", lv.bc[2 * d + 1] == "D")
    return S, Lm


def extended_gather(lv, r):
    """R_e r for every element: the pbar^3 window of the assembled residual (Sec. 2.2.2, eq 4).

    The window of element (ex,ey,ez) is the lattice box I in [ex p - 1, ex p + p + 1] (and
    likewise for J, K); points outside the domain read 0.  Returns (E, pbar, pbar, pbar).
    """
    p = lv.p
    pb = p + 3
    NX, NY, NZ = lv.lattice
    rg = to_global(lv, r).reshape(NZ, NY, NX)
    pad = np.zeros((NZ + 2, NY + 2, NX + 2))
    pad[1:-1, 1:-1, 1:-1] = rg
    nx, ny, nz = lv.nel
    out = np.empty((lv.E, pb, pb, pb))
    for e in range(lv.E):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        # padded index = lattice index + 1; window starts at lattice ex p - 1
        out[e] = pad[ez * p:ez * p + pb, ey * p:ey * p + pb, ex * p:ex * p + pb]
    return out


def fdm_apply(S, Lm, rbar):
    """Abar^-1 rbar = (S_z x S_y x S_x) D^-1 (S_z^T x S_y^T x S_x^T) rbar (eqs 8-9), per element,
    with D = I x I x Lambda_x + I x Lambda_y x I + Lambda_z x I x I."""
    Sx, Sy, Sz = S[:, 0], S[:, 1], S[:, 2]
    t = np.einsum("eia,ekji->ekja", Sx, rbar)           # S_x^T along r
    t = np.einsum("ejb,ekji->ekbi", Sy, t)              # S_y^T along s
    t = np.einsum("ekc,ekji->ecji", Sz, t)              # S_z^T along t
    Dg = Lm[:, 2][:, :, None, None] + Lm[:, 1][:, None, :, None] + Lm[:, 0][:, None, None, :]
    t = t / Dg
    t = np.einsum("eai,ekji->ekja", Sx, t)              # S_x along r
    t = np.einsum("ebj,ekji->ekbi", Sy, t)              # S_y along s
    return np.einsum("eck,ekji->ecji", Sz, t)           # S_z along t


def ras(lv, r):
    """Restrictive additive Schwarz (Sec. 2.2.2, after eq 9): only each element's own nodes of
    its local solve are kept, weighted by 1/(number of elements sharing the node), then summed.
    READING: 'changing W_e' is the partition-of-unity weight 1/mult on own nodes, 0 on overlap."""
    S, Lm = lv.extra["fdm"]
    z = fdm_apply(S, Lm, extended_gather(lv, r))
    p = lv.p
    own = z[:, 1:p + 2, 1:p + 2, 1:p + 2]
    return lv.mask * qqt(lv, own / lv.mult)


def asm(lv, r):
    """Additive Schwarz, eq 4: s = W sum_e R_e^T Abar_e^-1 R_e r with W post-multiplying by the
    inverse of the number of subdomains covering each node (Sec. 2.2.2)."""
    S, Lm = lv.extra["fdm"]
    z = fdm_apply(S, Lm, extended_gather(lv, r))
    p = lv.p
    pb = p + 3
    NX, NY, NZ = lv.lattice
    acc = np.zeros((NZ + 2, NY + 2, NX + 2))
    cnt = np.zeros((NZ + 2, NY + 2, NX + 2))
    nx, ny, nz = lv.nel
    for e in range(lv.E):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        sl = (slice(ez * p, ez * p + pb), slice(ey * p, ey * p + pb), slice(ex * p, ex * p + pb))
        acc[sl] += z[e]
        cnt[sl] += 1.0
    s = (acc / cnt)[1:-1, 1:-1, 1:-1].reshape(-1)
    return lv.mask * from_global(lv, s)


def jacobi(lv, r):
    """Jacobi surrogate S = diag(A)^-1 (Sec. 2.2.3)."""
    return lv.mask * r / lv.extra["diag"]


# =============================================================================================
# Chebyshev acceleration (Sec. 2.2.3, Algorithm 2) and the Arnoldi bound estimate.
# =============================================================================================


def chebyshev(res, A, S, lmin, lmax, order):
    """Algorithm 2 applied to the residual ``res`` = b - A x; returns the correction.

    theta, delta, sigma = theta/delta, rho_1 = 1/sigma; r = S res, d_1 = r/theta, x_1 = 0;
    for k = 1..order: x += d_k; r -= S A d_k; rho_{k+1} = 1/(2 sigma - rho_k);
    d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) r; then a final x += d.
    READING: the final update uses d_{order+1}, so the error polynomial has degree order+1.
    """
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = S(res)
    d = r / theta
    x = np.zeros_like(res)
    for _ in range(order):
        x = x + d
        r = r - S(A(d))
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x + d


def arnoldi_lambda(A, S, v0, dotf, steps=10):
    """lambda-tilde: largest |Ritz value| after ``steps`` rounds of Arnoldi (modified
    Gram-Schmidt) on S A (Sec. 2.2.3).  Stops early if the Krylov space is exhausted
    (subdiagonal <= 1e-12 of the largest |H| entry)."""
    v = v0 / math.sqrt(dotf(v0, v0))
    Vs = [v]
    H = np.zeros((steps + 1, steps))
    m = steps
    for j in range(steps):
        w = S(A(Vs[j]))
        for i in range(j + 1):
            H[i, j] = dotf(w, Vs[i])
            w = w - H[i, j] * Vs[i]
        H[j + 1, j] = math.sqrt(max(dotf(w, w), 0.0))
        if H[j + 1, j] <= 1e-12 * np.max(np.abs(H[:j + 2, :j + 1])):
            m = j + 1
            break
        Vs.append(w / H[j + 1, j])
    ritz = np.linalg.eigvals(H[:m, :m])
    return float(np.max(np.abs(ritz))), H[:m + 1, :m]


# =============================================================================================
# p-multigrid (Sec. 2.2.2, Algorithm 1): transfers, coarse solve, V-cycle.
# =============================================================================================


def interp_1d(p_fine, p_coarse):
    """J_ij = h^c_j(xi^f_i): coarse GLL basis evaluated at the fine GLL points."""
    xf, _ = gll(p_fine)
    xc, _ = gll(p_coarse)
    return lagrange_eval(xc, xf)


def prolong(lf, lc, ec):
    """P e_c = (J x J x J) e_c element by element (continuous in, continuous out)."""
    J = interp_1d(lf.p, lc.p)
    return along_t(J, along_s(J, along_r(J, ec)))


def restrict(lf, lc, rf):
    """P^T r_f in L-vector form: M_c QQ^T_c (J^T x J^T x J^T)(r_f / mult_f).
    For a continuous r_f this is the transpose of the global prolongation."""
    J = interp_1d(lf.p, lc.p)
    t = rf / lf.mult
    return lc.mask * qqt(lc, along_t(J.T, along_s(J.T, along_r(J.T, t))))


def pcg(A, Minv, b, dotf, tol, maxit):
    """Preconditioned conjugate gradients (textbook), x0 = 0, stop when ||r|| <= tol ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    r0 = math.sqrt(dotf(r, r))
    if r0 == 0.0:
        return x, 0
    z = Minv(r)
    pv = z.copy()
    rz = dotf(r, z)
    for it in range(1, maxit + 1):
        w = A(pv)
        alpha = rz / dotf(pv, w)
        x = x + alpha * pv
        r = r - alpha * w
        if math.sqrt(dotf(r, r)) <= tol * r0:
            return x, it
        z = Minv(r)
        rz_new = dotf(r, z)
        beta = rz_new / rz
        rz = rz_new
        pv = z + beta * pv
    return x, maxit


@dataclass
class PMG:
    levels: list
    smoother: str            # 'ras', 'asm' or 'jacobi'
    order: list              # Chebyshev order per level (coarsest unused)
    bounds: list             # (lmin, lmax) per level
    lam: list                # lambda-tilde per level
    coarse_tol: float = 1e-2
    coarse_maxit: int = 500
    coarse_iters: list = field(default_factory=list)
    cycle: str = "mult"      # 'mult' (Algorithm 1) or 'additive' (Sec. 2.2.2, no Chebyshev)


def smoother_op(pmg, l):
    lv = pmg.levels[l]
    if pmg.smoother == "ras":
        return lambda r: ras(lv, r)
    if pmg.smoother == "asm":
        return lambda r: asm(lv, r)
    return lambda r: jacobi(lv, r)


def pmg_setup(V, nel, schedule, smoother="ras", order=2, bc=("D",) * 6, amp=0.05,
              eig_lo=0.1, eig_hi=1.1, arnoldi_steps=10, seed=0, coarse_tol=1e-2, coarse_maxit=500,
              start_vectors=None, cycle="mult"):
    """Levels of the schedule, smoother data and Chebyshev bounds (Secs. 2.2.2-2.2.3).

    READING: every level is rediscretised on the same mapped mesh at its own order (geometry
    from the map evaluated at that level's GLL points).  Bounds (lmin, lmax) = (eig_lo, eig_hi)
    lambda-tilde (Sec. 2.2.3).  ``start_vectors[l]`` is the global start vector of level l
    (from workloads.arnoldi_start_global).
    """
    from workloads import arnoldi_start_global, arnoldi_seed  # seeded inputs only
    levels = [make_level(V, nel, p, bc, amp) for p in schedule]
    orders = order if isinstance(order, (list, tuple)) else [order] * len(levels)
    for lv in levels:
        lv.extra["diag"] = jacobi_diag(lv)
    pmg = PMG(levels=levels, smoother=smoother, order=list(orders), bounds=[], lam=[],
              coarse_tol=coarse_tol, coarse_maxit=coarse_maxit, cycle=cycle)
    for l, lv in enumerate(levels[:-1]):
        if smoother in ("ras", "asm"):
            lv.extra["fdm"] = fdm_setup(lv, V, amp)
        if start_vectors is not None:
            vg = start_vectors[l]
        else:
            vg = arnoldi_start_global(arnoldi_seed(seed, l), lv.n_global)
        v0 = lv.mask * from_global(lv, vg)
        lam, _ = arnoldi_lambda(lambda u, lv=lv: ax(lv, u), smoother_op(pmg, l), v0,
                                lambda a, b, lv=lv: dot(lv, a, b), arnoldi_steps)
        pmg.lam.append(lam)
        pmg.bounds.append((eig_lo * lam, eig_hi * lam))
    return pmg


def coarse_solve(pmg, b):
    """Coarsest level (p = 1): Jacobi-PCG to relative residual coarse_tol (default 1e-2).
    READING: replaces the paper's single BoomerAMG V-cycle (Sec. 2.2.2), which needs a
    third-party AMG library; like one AMG cycle it is an inexact solve (a residual reduction
    of about two orders), not a solve to rounding."""
    lv = pmg.levels[-1]
    x, it = pcg(lambda u: ax(lv, u), lambda r: jacobi(lv, r), b,
                lambda a, c: dot(lv, a, c), pmg.coarse_tol, pmg.coarse_maxit)
    pmg.coarse_iters.append(it)
    return x


def vcycle_additive(pmg, b, l=0):
    """Additive V-cycle (Sec. 2.2.2): with ASM or RAS smoothers without Chebyshev acceleration
    the paper applies the smoother and the coarse correction to the same residual, with no
    post-smoothing, so that the residual is not re-evaluated:  x = S b + P V(P^T b).
    READING: S is the smoother itself (no Chebyshev polynomial, no 1/theta scaling); the same
    rule applies on every level, the coarsest solved as in Algorithm 1."""
    if l == len(pmg.levels) - 1:
        return coarse_solve(pmg, b)
    lv, lc = pmg.levels[l], pmg.levels[l + 1]
    x = smoother_op(pmg, l)(b)                                # smooth the residual itself
    ec = vcycle_additive(pmg, restrict(lv, lc, b), l + 1)     # coarse correction of the same b
    return x + prolong(lv, lc, ec)


def vcycle(pmg, b, l=0):
    """Algorithm 1 with x = 0 on entry; M is the Chebyshev-accelerated smoother of Algorithm 2.
    A preconditioner set up with cycle='additive' runs vcycle_additive instead."""
    if pmg.cycle == "additive":
        return vcycle_additive(pmg, b, l)
    if l == len(pmg.levels) - 1:
        return coarse_solve(pmg, b)
    lv = pmg.levels[l]
    A = lambda u: ax(lv, u)
    S = smoother_op(pmg, l)
    lmin, lmax = pmg.bounds[l]
    k = pmg.order[l]
    x = chebyshev(b, A, S, lmin, lmax, k)                     # x = 0 + M(b - A 0)
    r = b - A(x)                                              # re-evaluate residual
    rc = restrict(lv, pmg.levels[l + 1], r)                   # coarsen
    ec = vcycle(pmg, rc, l + 1)                               # solve / recurse
    x = x + prolong(lv, pmg.levels[l + 1], ec)                # prolongate, update
    x = x + chebyshev(b - A(x), A, S, lmin, lmax, k)          # post-smoothing
    return x


# =============================================================================================
# Outer Krylov methods (Sec. 2.2): flexible CG and right-preconditioned flexible GMRES.
# =============================================================================================


def fpcg(A, M, b, x0, dotf, tol=1e-8, maxit=1000):
    """Flexible PCG with beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k); stop when
    ||r_k|| <= tol ||r_0|| (unique-node 2-norm).  Returns (x, iterations, rel. residual)."""
    x = x0.copy()
    r = b - A(x)
    r0 = math.sqrt(dotf(r, r))
    if r0 == 0.0:
        return x, 0, 0.0
    z = M(r)
    pv = z.copy()
    rz = dotf(r, z)
    rel = 1.0
    for it in range(1, maxit + 1):
        w = A(pv)
        alpha = rz / dotf(pv, w)
        x = x + alpha * pv
        r_new = r - alpha * w
        rel = math.sqrt(dotf(r_new, r_new)) / r0
        if rel <= tol:
            return x, it, rel
        z_new = M(r_new)
        rz_new = dotf(z_new, r_new)
        beta = (rz_new - dotf(z_new, r)) / rz
        r, z, rz = r_new, z_new, rz_new
        pv = z + beta * pv
    return x, maxit, rel


def fgmres(A, M, b, x0, dotf, m=20, tol=1e-8, maxit=1000):
    """Restarted flexible GMRES(m), right preconditioned, modified Gram-Schmidt, Givens
    rotations; stop when the residual estimate <= tol ||r_0||.  Returns (x, iters, rel)."""
    x = x0.copy()
    r = b - A(x)
    r0 = math.sqrt(dotf(r, r))
    if r0 == 0.0:
        return x, 0, 0.0
    total = 0
    beta = r0
    rel = 1.0
    while total < maxit:
        Vs = [r / beta]
        Zs = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j_used = 0
        for j in range(m):
            z = M(Vs[j])
            Zs.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = dotf(w, Vs[i])
                w = w - H[i, j] * Vs[i]
            H[j + 1, j] = math.sqrt(dotf(w, w))
            Vs.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_used = j + 1
            rel = abs(g[j + 1]) / r0
            if rel <= tol or total >= maxit:
                break
        y = np.zeros(j_used)
        for i in range(j_used - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_used] @ y[i + 1:]) / H[i, i]
        for i in range(j_used):
            x = x + y[i] * Zs[i]
        if rel <= tol:
            break
        r = b - A(x)
        beta = math.sqrt(dotf(r, r))
    return x, total, rel


# =============================================================================================
# Projection onto prior solutions (Secs. 3.2 and 4.2): the initial guess for a new right-hand
# side is the element of span{x_1..x_m} closest to A^-1 b in the A-norm.
# =============================================================================================


def projection_guess(lv, xs, b):
    """The A-orthogonal projection of A^-1 b onto span(xs), by its definition: xbar = X a with the
    Galerkin system (x_i, A x_j) a_j = (x_i, b) (inner products counting each global node once),
    solved by least squares so that a dependent set still defines the same projection."""
    if not xs:
        return np.zeros_like(b)
    Ax = [ax(lv, x) for x in xs]
    G = np.array([[dot(lv, xi, Axj) for Axj in Ax] for xi in xs])
    c = np.array([dot(lv, xi, b) for xi in xs])
    a = np.linalg.lstsq(G, c, rcond=1e-13)[0]
    return sum(ai * xi for ai, xi in zip(a, xs))


# =============================================================================================
# Convenience: whole problem set-up and solve (used by tests and the cpu baseline).
# =============================================================================================


def problem(V, nel, p, bc=("D",) * 6, amp=0.05, f=None):
    """Fine level and right-hand side b = M QQ^T B_L f for f evaluated at the nodes."""
    lv = make_level(V, nel, p, bc, amp)
    if f is None:
        from workloads import f_rhs
        f = f_rhs
    b = rhs(lv, f(lv.X[0], lv.X[1], lv.X[2]))
    return lv, b


def solve(lv, b, pmg=None, method="fpcg", tol=1e-8, maxit=1000, restart=20):
    """Outer solve with pMG (if given) or Jacobi preconditioning; x0 = 0."""
    A = lambda u: ax(lv, u)
    if pmg is None:
        d = jacobi_diag(lv)
        M = lambda r: lv.mask * r / d
    else:
        M = lambda r: vcycle(pmg, r)
    dotf = lambda a, c: dot(lv, a, c)
    x0 = np.zeros_like(b)
    if method == "fpcg":
        return fpcg(A, M, b, x0, dotf, tol, maxit)
    return fgmres(A, M, b, x0, dotf, restart, tol, maxit)
