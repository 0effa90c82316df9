"""Parity at the benchmark size: 32^3 elements, p = 7, perturbed lattice seed 0, pMG 7-5-3-1
Cheby-RAS(2), the configuration bench.py times.

The oracle cannot run the whole problem in seconds, so it checks sampled outputs it can compute
element by element (local Ax, extension gather, FDM, RAS at element-interior nodes,
prolongation), using one-element or 3x3x3-element pieces of the same lattice (the geometry and
box lengths of an element depend only on its own and its face neighbours' vertices), and the
solve is checked through properties that hold at any size: symmetry of A, the unique-node inner
product of lattice functions, convergence to the tolerance with the true residual, determinism,
graph solve equal to the host-driven solve.
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import gpu, rel_err

pytestmark = pytest.mark.gpu

NEL, P, SCHED = (32, 32, 32), 7, (7, 5, 3, 1)
SAMPLE = [0, 31, 32 * 32 - 1, 16 + 32 * (16 + 32 * 16), 5 + 32 * (31 + 32 * 9), 32 ** 3 - 1]


@pytest.fixture(scope="module")
def big():
    torch, se = gpu()
    m = se.se_mesh_create(NEL, P, perturb_frac=0.05, seed=0, deform_amp=wl.DEFORM_AMP)
    P_ = se.se_pmg_setup(m, se.pmg_desc(SCHED, se.SE_SMOOTH_RAS, 2))
    V = wl.vertex_lattice(NEL, 0.05, 0)
    info = se.se_mesh_get_info(m)
    yield torch, se, m, P_, V, info
    se.se_pmg_destroy(P_)
    se.se_mesh_destroy(m)


def coords(e, nel=NEL):
    nx, ny, _ = nel
    return e % nx, (e // nx) % ny, e // (nx * ny)


def piece(V, e, p, halo):
    """Oracle level of the elements around e (halo 0: e alone; 1: up to 3x3x3, clipped) and the
    index of e inside it."""
    ex, ey, ez = coords(e)
    lo = [max(c - halo, 0) for c in (ex, ey, ez)]
    hi = [min(c + halo, n - 1) for c, n in zip((ex, ey, ez), NEL)]
    sub = V[lo[2]:hi[2] + 2, lo[1]:hi[1] + 2, lo[0]:hi[0] + 2]
    nel = (hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1)
    lv = o.make_level(sub, nel, p, amp=wl.DEFORM_AMP)
    le = (ex - lo[0]) + nel[0] * ((ey - lo[1]) + nel[1] * (ez - lo[2]))
    return lv, le, sub, nel


def global_ids(p, nel=NEL):
    I, J, K = o.lattice_indices(nel, p)
    NX, NY = nel[0] * p + 1, nel[1] * p + 1
    return I, J, K, NX, NY


def test_sampled_local_ax(big):
    torch, se, m, P_, V, info = big
    N3 = (P + 1) ** 3
    u = torch.from_numpy(wl.random_lvector(info.L, 11)).cuda()
    y = torch.empty_like(u)
    se.se_ax(m, u, y, 0)
    un, yn = u.cpu().numpy(), y.cpu().numpy()
    for e in SAMPLE:
        lv, le, _, _ = piece(V, e, P, 0)
        ue = un[e * N3:(e + 1) * N3].reshape(1, P + 1, P + 1, P + 1)
        ref = o.ax_local(lv, ue)
        assert rel_err(yn[e * N3:(e + 1) * N3], ref.reshape(-1)) <= 1e-12


def test_symmetry_and_unique_node_dot(big):
    torch, se, m, P_, V, info = big
    I, J, K, NX, NY = global_ids(P)
    NZ = NEL[2] * P + 1
    fa = lambda I, J, K: np.sin(0.011 * I + 0.3) * np.cos(0.017 * J) + 0.001 * K
    fb = lambda I, J, K: np.cos(0.005 * I * J / 7.0) - 0.002 * K
    to = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64).reshape(-1)).cuda()
    a, b = to(fa(I, J, K)), to(fb(I, J, K))
    d = se.se_dot(m, a, b)
    Ig, Jg, Kg = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ref = float(np.sum(fa(Ig, Jg, Kg) * fb(Ig, Jg, Kg)))
    assert abs(d - ref) <= 1e-12 * abs(ref)
    free = (I > 0) & (I < NX - 1) & (J > 0) & (J < NY - 1) & (K > 0) & (K < NZ - 1)
    a, b = to(np.where(free, fa(I, J, K), 0.0)), to(np.where(free, fb(I, J, K), 0.0))
    au, bu = torch.empty_like(a), torch.empty_like(b)
    se.se_ax(m, a, au)
    se.se_ax(m, b, bu)
    s1, s2 = se.se_dot(m, b, au), se.se_dot(m, a, bu)
    assert abs(s1 - s2) <= 1e-11 * max(abs(s1), 1.0)


def test_sampled_gather_fdm_ras_and_prolong(big):
    torch, se, m, P_, V, info = big
    pb = P + 3
    N3 = (P + 1) ** 3
    I, J, K, NX, NY = global_ids(P)
    NZ = NEL[2] * P + 1
    g = lambda I, J, K: np.sin(0.013 * I + 0.07 * J) * np.cos(0.019 * K) + 0.5
    free = (I > 0) & (I < NX - 1) & (J > 0) & (J < NY - 1) & (K > 0) & (K < NZ - 1)
    r = torch.from_numpy(np.ascontiguousarray(np.where(free, g(I, J, K), 0.0), dtype=np.float64).reshape(-1)).cuda()
    rbar = torch.empty(info.E * pb ** 3, dtype=torch.float64, device="cuda")
    se.se_pmg_gather_ext(P_, 0, r, rbar)
    rb = rbar.cpu().numpy().reshape(info.E, pb, pb, pb)
    zbar_in = torch.from_numpy(wl.random_lvector(info.E * pb ** 3, 12)).cuda()
    zbar = torch.empty_like(zbar_in)
    se.se_pmg_fdm(P_, 0, zbar_in, zbar)
    zi, zo = zbar_in.cpu().numpy().reshape(info.E, pb, pb, pb), zbar.cpu().numpy().reshape(info.E, pb, pb, pb)
    s = torch.empty_like(r)
    se.se_pmg_smooth(P_, 0, r, s)
    sn = s.cpu().numpy()
    for e in SAMPLE:
        ex, ey, ez = coords(e)
        # extension gather: lattice window with zeros outside the domain / on Dirichlet faces
        a_ = np.arange(pb) + ex * P - 1
        b_ = np.arange(pb) + ey * P - 1
        c_ = np.arange(pb) + ez * P - 1
        Cc, Bb, Aa = np.meshgrid(c_, b_, a_, indexing="ij")
        inside = (Aa > 0) & (Aa < NX - 1) & (Bb > 0) & (Bb < NY - 1) & (Cc > 0) & (Cc < NZ - 1)
        assert np.array_equal(rb[e], np.where(inside, g(Aa, Bb, Cc), 0.0))
        # FDM of the element with factors from a 3x3x3 piece
        lv, le, sub, nel = piece(V, e, P, 1)
        S, Lm = o.fdm_setup(lv, sub, amp=wl.DEFORM_AMP)
        ref = o.fdm_apply(S[le:le + 1], Lm[le:le + 1], zi[e:e + 1])[0]
        assert rel_err(zo[e], ref) <= 1e-10
        # RAS at element-interior nodes (one copy, no overlap from other windows): FDM own part
        zr = o.fdm_apply(S[le:le + 1], Lm[le:le + 1], rb[e:e + 1])[0][1:P + 2, 1:P + 2, 1:P + 2]
        got = sn[e * N3:(e + 1) * N3].reshape(P + 1, P + 1, P + 1)
        assert rel_err(got[2:P - 1, 2:P - 1, 2:P - 1], zr[2:P - 1, 2:P - 1, 2:P - 1]) <= 1e-10
    # prolongation 5 -> 7 of a coarse lattice function, element by element
    Pc = 5
    Ic, Jc, Kc, NXc, NYc = global_ids(Pc)
    info_c = se.se_pmg_level_info(P_, 1)
    ec = torch.from_numpy(np.ascontiguousarray(g(Ic, Jc, Kc), dtype=np.float64).reshape(-1)).cuda()
    ef = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_pmg_prolong(P_, 0, ec, ef)
    ecn, efn = ec.cpu().numpy(), ef.cpu().numpy()
    Jm = o.interp_1d(P, Pc)
    Nc3 = (Pc + 1) ** 3
    for e in SAMPLE:
        ee = ecn[e * Nc3:(e + 1) * Nc3].reshape(Pc + 1, Pc + 1, Pc + 1)
        ref = o.along_t(Jm, o.along_s(Jm, o.along_r(Jm, ee)))
        assert rel_err(efn[e * N3:(e + 1) * N3].reshape(P + 1, P + 1, P + 1), ref) <= 1e-13
    assert info_c.L == info.E * Nc3


def test_full_solve_converges_and_is_deterministic(big):
    torch, se, m, P_, V, info = big
    xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, -1)
    f = 3 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    b = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_rhs(m, f.contiguous(), b)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    s1 = se.se_solve(m, P_, b, x1, tol=1e-8)
    s2 = se.se_solve(m, P_, b, x2, tol=1e-8, graph_capture=1)
    assert s1.rel_residual <= 1e-8 and s1.iterations == s2.iterations
    assert torch.equal(x1, x2)
    w = torch.empty_like(b)
    se.se_ax(m, x1, w)
    r = b - w
    assert math.sqrt(se.se_dot(m, r, r) / se.se_dot(m, b, b)) <= 1.5e-8
    # discretisation error against u* at p = 7 on the 32^3 mesh
    ustar = torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    assert float((x1 - ustar).abs().max()) < 1e-6
