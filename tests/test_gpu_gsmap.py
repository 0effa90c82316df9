"""GPU parity of QQ^T driven by the sorted index map (Sec. 2.1, direct stiffness summation),
through the C ABI: the standalone se_gsmap handle on lattice and on arbitrary connectivities,
and meshes created with SE_MESH_GS_MAP (every QQ^T of the mesh and of its preconditioner levels
through the map) against the oracle and against the default direction sweeps.

Tolerances: the map sums the copies of a node in ascending local-id order from the first, the
order in which the oracle's histogram sum (numpy bincount) adds them, so FP64 results are
compared for exact equality; FP32 within (m - 1) 2^-24 times the sum of |u| over the m copies.
The sweeps add copies in another order, so map against sweeps is within 1e-14 of the largest
entry; solves meet the solve tests' bars (iterations within one of the oracle's, solution 1e-5).
"""
import math

import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, gpu, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [((1, 1, 1), 2), ((3, 2, 4), 3), ((2, 3, 2), 5), ((2, 2, 2), 7), ((3, 1, 2), 10)]
BCS = [("D",) * 6, ("N", "D", "N", "N", "D", "N")]


def qqt_reference(gid, u, dirichlet=None, mask=True):
    """Sum over the copies of each global id in local-id order (numpy bincount), then the mask."""
    gid = np.asarray(gid).ravel()
    s = np.bincount(gid, weights=u.ravel())[gid]
    if mask and dirichlet is not None:
        masked = np.zeros(gid.max() + 1, dtype=bool)
        np.logical_or.at(masked, gid, np.asarray(dirichlet).ravel() != 0)
        s = np.where(masked[gid], 0.0, s)
    return s


def check_fp32(torch, se, g, gid, u, dirichlet):
    t = torch.from_numpy(u.astype(np.float32)).cuda()
    se.se_gsmap_apply(g, t, 1)
    got = t.cpu().numpy().astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    ref = qqt_reference(gid, u32, dirichlet)
    cnt = np.bincount(gid)[gid]
    bound = (cnt - 1) * 2.0 ** -24 * qqt_reference(gid, np.abs(u32)) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("nel,p", SHAPES)
@pytest.mark.parametrize("bc", BCS)
def test_handle_on_lattice_numbering_equals_oracle(nel, p, bc):
    torch, se = gpu()
    lv = o.make_level(wl.vertex_lattice(nel, 0.05, p), nel, p, bc)
    gid = lv.gid.ravel()
    dirichlet = (lv.mask.ravel() == 0).astype(np.uint8)
    g = se.se_gsmap_create(gid, dirichlet)
    try:
        assert se.se_gsmap_info(g) == se.se_gsmap_count(gid, dirichlet)
        u = wl.random_lvector(gid.size, 100 + p)
        for mask in (0, 1):
            t = torch.from_numpy(u.copy()).cuda()
            se.se_gsmap_apply(g, t, mask)
            ref = o.qqt(lv, u.reshape(lv.gid.shape)).ravel()
            if mask:
                ref = ref * lv.mask.ravel()
            assert np.array_equal(t.cpu().numpy(), ref)
        check_fp32(torch, se, g, gid, u, dirichlet)
    finally:
        se.se_gsmap_destroy(g)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_handle_on_arbitrary_connectivity(seed):
    """Multiplicities 1..12 in random positions: every bucket, including the general one."""
    torch, se = gpu()
    rng = np.random.default_rng(seed)
    n_global = [3000, 40000, 7, 1][seed]
    mult = rng.integers(1, 13, size=n_global)
    gid = np.repeat(np.arange(n_global), mult)
    rng.shuffle(gid)
    if seed == 2:
        gid = gid * 1000003 + 10 ** 12  # sparse labels
    dirichlet = (rng.random(gid.size) < 0.1).astype(np.uint8)
    g = se.se_gsmap_create(gid, dirichlet)
    try:
        u = wl.random_lvector(gid.size, 7 + seed)
        _, comp = np.unique(gid, return_inverse=True)
        for mask in (0, 1):
            t = torch.from_numpy(u.copy()).cuda()
            se.se_gsmap_apply(g, t, mask)
            assert np.array_equal(t.cpu().numpy(), qqt_reference(comp, u, dirichlet, bool(mask)))
        check_fp32(torch, se, g, comp, u, dirichlet)
    finally:
        se.se_gsmap_destroy(g)


@pytest.mark.parametrize("case", ["one_node_1000_copies", "single_point", "single_masked_point",
                                  "no_shared_node"])
def test_handle_degenerate_maps(case):
    """Degenerate numberings: one global node shared by every local point (one CSR group of 1000
    copies), a single local point with and without the Dirichlet flag, and no shared node."""
    torch, se = gpu()
    gid, dirichlet = {
        "one_node_1000_copies": (np.zeros(1000, dtype=np.int64), None),
        "single_point": (np.array([7]), None),
        "single_masked_point": (np.array([7]), np.array([1], dtype=np.uint8)),
        "no_shared_node": (np.arange(50) * 3, (np.arange(50) % 2).astype(np.uint8)),
    }[case]
    g = se.se_gsmap_create(gid, dirichlet)
    try:
        assert se.se_gsmap_info(g) == se.se_gsmap_count(gid, dirichlet)
        u = wl.random_lvector(gid.size, 3)
        _, comp = np.unique(gid, return_inverse=True)
        for mask in (0, 1):
            t = torch.from_numpy(u.copy()).cuda()
            se.se_gsmap_apply(g, t, mask)
            assert np.array_equal(t.cpu().numpy(), qqt_reference(comp, u, dirichlet, bool(mask)))
    finally:
        se.se_gsmap_destroy(g)


def gpu_problem(c):
    xyz = c.empty(3 * c.info.L)
    c.se.se_mesh_nodes(c.m, xyz)
    X = xyz.cpu().numpy().reshape(3, -1)
    b = c.empty()
    c.se.se_mesh_rhs(c.m, c.to_gpu(wl.f_rhs(X[0], X[1], X[2])), b)
    return b


@pytest.mark.parametrize("nel,p,bc", [((3, 2, 4), 3, BCS[0]), ((2, 2, 2), 7, BCS[1])])
def test_mesh_flag_operator(nel, p, bc):
    cm = Case(nel, p, seed=3, bc=bc, flags=2)  # SE_MESH_GS_MAP
    cs = Case(nel, p, seed=3, bc=bc)
    se = cm.se
    assert se.SE_MESH_GS_MAP == 2
    try:
        u = wl.random_lvector(cm.info.L, 5)
        for mask in (0, 1):
            t = cm.to_gpu(u)
            se.se_gs(cm.m, t, mask)
            ref = o.qqt(cm.lv, u.reshape(cm.lv.gid.shape))
            if mask:
                ref = ref * cm.lv.mask
            assert np.array_equal(cm.to_np(t), ref)
            ts = cs.to_gpu(u)
            se.se_gs(cs.m, ts, mask)
            assert rel_err(cm.to_np(t), cs.to_np(ts)) <= 1e-14
        v = cm.to_gpu(cm.random_continuous(9))
        ym, ys = cm.empty(), cs.empty()
        se.se_ax(cm.m, v, ym)
        se.se_ax(cs.m, v, ys)
        assert rel_err(cm.to_np(ym), cs.to_np(ys)) <= 1e-14
        assert rel_err(cm.to_np(ym), o.ax(cm.lv, cm.to_np(v))) <= 1e-12
    finally:
        cm.close()
        cs.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mesh_flag_solve(precision):
    """pMG 7-3-1 Cheby-RAS(2) FPCG on the 4^3 p = 7 box with every QQ^T through the map."""
    c = Case((4, 4, 4), 7, pert=0.0, flags=2)
    se = c.se
    prec = se.SE_FP64 if precision == "fp64" else se.SE_FP32
    P = se.se_pmg_setup(c.m, se.pmg_desc((7, 3, 1), se.SE_SMOOTH_RAS, 2, precision=prec))
    try:
        b = gpu_problem(c)
        lvo, bo = o.problem(c.V, c.nel, c.p, amp=c.amp)
        assert rel_err(c.to_np(b), bo) <= 1e-13
        x, xg = c.empty().zero_(), c.empty().zero_()
        st = se.se_solve(c.m, P, b, x, tol=1e-8)
        sg = se.se_solve(c.m, P, b, xg, tol=1e-8, graph_capture=1)
        assert sg.iterations == st.iterations and np.array_equal(c.to_np(x), c.to_np(xg))
        pmg = o.pmg_setup(c.V, c.nel, (7, 3, 1), smoother="ras", order=2, amp=c.amp)
        xo, it_o, _ = o.solve(lvo, bo, pmg, tol=1e-8)
        assert abs(st.iterations - it_o) <= 1, (st.iterations, it_o)
        r = bo - o.ax(c.lv, c.to_np(x))
        assert math.sqrt(o.dot(c.lv, r, r) / o.dot(c.lv, bo, bo)) <= 1.5e-8
        assert rel_err(c.to_np(x), xo) <= 1e-5
    finally:
        se.se_pmg_destroy(P)
        c.close()


def test_bench_size_map_equals_sweeps():
    """32^3 elements, p = 7 (the benchmark mesh): QQ^T by the map and by the sweeps agree, and
    the benchmark's solve (pMG 7-5-3-1 Cheby-Jac(1), FPCG to 1e-8) on the map mesh takes the
    sweep mesh's iteration count and reaches the tolerance."""
    torch, se = gpu()
    nel, p = (32, 32, 32), 7
    mm = se.se_mesh_create(nel, p, perturb_frac=0.05, seed=0, deform_amp=wl.DEFORM_AMP, flags=2)
    ms = se.se_mesh_create(nel, p, perturb_frac=0.05, seed=0, deform_amp=wl.DEFORM_AMP)
    Pm = Ps = None
    try:
        L = se.se_mesh_get_info(mm).L
        gen = torch.Generator(device="cuda").manual_seed(0)
        u = torch.rand(L, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
        a, b_ = u.clone(), u.clone()
        se.se_gs(mm, a, 1)
        se.se_gs(ms, b_, 1)
        assert float((a - b_).abs().max()) <= 1e-14 * float(b_.abs().max())
        xyz = torch.empty(3 * L, dtype=torch.float64, device="cuda")
        se.se_mesh_nodes(ms, xyz)
        X = xyz.view(3, L)
        f = (3 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1])
             * torch.sin(math.pi * X[2])).contiguous()
        bm, bs = torch.empty_like(u), torch.empty_like(u)
        se.se_mesh_rhs(mm, f, bm)
        se.se_mesh_rhs(ms, f, bs)
        assert float((bm - bs).abs().max()) <= 1e-14 * float(bs.abs().max())
        desc = se.pmg_desc((7, 5, 3, 1), se.SE_SMOOTH_JACOBI, 1)
        Pm, Ps = se.se_pmg_setup(mm, desc), se.se_pmg_setup(ms, desc)
        xm, xs = torch.zeros_like(u), torch.zeros_like(u)
        stm = se.se_solve(mm, Pm, bs, xm, tol=1e-8, graph_capture=1)
        sts = se.se_solve(ms, Ps, bs, xs, tol=1e-8, graph_capture=1)
        assert abs(stm.iterations - sts.iterations) <= 1 and stm.rel_residual <= 1e-8
        assert float((xm - xs).abs().max()) <= 1e-6 * float(xs.abs().max())
    finally:
        for P in (Pm, Ps):
            if P:
                se.se_pmg_destroy(P)
        se.se_mesh_destroy(mm)
        se.se_mesh_destroy(ms)
