"""GPU parity of the operator path (Sec. 2.1) against the oracle, through the C ABI.

Tolerances: FP64 operator relative error <= 1e-12 (max-norm relative to the largest entry);
FP32 operator <= 2e-5 (single precision with O(N) accumulation depth).
"""
import numpy as np
import pytest

import oracle as o
import workloads as wl
from tests.gpu_common import Case, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [((1, 1, 1), 1), ((2, 3, 1), 2), ((3, 2, 2), 3), ((2, 2, 3), 4), ((3, 3, 2), 5),
          ((2, 2, 2), 6), ((3, 1, 2), 7), ((2, 2, 2), 8), ((1, 2, 2), 9), ((2, 1, 1), 10)]


@pytest.mark.parametrize("nel,p", SHAPES)
def test_geometry_and_vertices(nel, p):
    c = Case(nel, p, seed=p)
    try:
        xyz = c.empty(3 * c.info.L)
        c.se.se_mesh_nodes(c.m, xyz)
        X = xyz.cpu().numpy().reshape(c.lv.X.shape)
        assert rel_err(X, c.lv.X) < 1e-14
        assert c.info.E == np.prod(nel) and c.info.n_dof == np.prod(nel) * p ** 3
        assert c.info.n_global == c.lv.n_global
    finally:
        c.close()


def test_library_vertex_generator_matches_inputs():
    torch, se = Case((1, 1, 1), 1).torch, Case((1, 1, 1), 1).se
    nel = (5, 4, 3)
    m = se.se_mesh_create(nel, 3, perturb_frac=0.05, seed=11)
    try:
        out = np.empty((nel[2] + 1) * (nel[1] + 1) * (nel[0] + 1) * 3)
        se.se_mesh_vertices(m, out)
        ref = wl.vertex_lattice(nel, 0.05, seed=11).reshape(-1)
        assert np.array_equal(out, ref)
    finally:
        se.se_mesh_destroy(m)


@pytest.mark.parametrize("nel,p", SHAPES)
@pytest.mark.parametrize("bc", [("D",) * 6, ("N", "D", "N", "N", "D", "N")])
def test_ax_fp64(nel, p, bc):
    c = Case(nel, p, seed=10 + p, bc=bc)
    try:
        u = c.random_continuous(1, masked=False)
        y = c.empty()
        ug = c.to_gpu(u)
        se = c.se
        # assembled + masked
        se.se_ax(c.m, ug, y, se.SE_AX_ASSEMBLE | se.SE_AX_MASK)
        assert rel_err(c.to_np(y), o.ax(c.lv, u)) <= 1e-12
        # local only
        se.se_ax(c.m, ug, y, 0)
        assert rel_err(c.to_np(y), o.ax_local(c.lv, u)) <= 1e-12
        # assembled without mask
        se.se_ax(c.m, ug, y, se.SE_AX_ASSEMBLE)
        assert rel_err(c.to_np(y), o.ax(c.lv, u, mask=False)) <= 1e-12
        # FP32 compute path
        se.se_ax(c.m, ug, y, se.SE_AX_ASSEMBLE | se.SE_AX_MASK | se.SE_AX_FP32)
        assert rel_err(c.to_np(y), o.ax(c.lv, u)) <= 2e-5
    finally:
        c.close()


@pytest.mark.parametrize("nel,p", [((1, 1, 1), 1), ((3, 2, 2), 3), ((3, 3, 2), 5), ((3, 1, 2), 7),
                                   ((1, 2, 2), 9), ((7, 5, 3), 3), ((4, 4, 5), 7)])
def test_ax_fp32_pipelined_path(nel, p):
    # FP32, no input mask, even N: the TMA-pipelined kernel (groups, ragged last group)
    c = Case(nel, p, seed=30 + p)
    try:
        u = c.random_continuous(4, masked=False)
        y = c.empty()
        se = c.se
        se.se_ax(c.m, c.to_gpu(u), y, se.SE_AX_FP32)
        assert rel_err(c.to_np(y), o.ax_local(c.lv, u)) <= 2e-5
        se.se_ax(c.m, c.to_gpu(u), y, se.SE_AX_FP32 | se.SE_AX_ASSEMBLE)
        assert rel_err(c.to_np(y), o.ax(c.lv, u, mask=False)) <= 2e-5
    finally:
        c.close()


def test_neumann_nullspace_and_symmetry_on_gpu():
    c = Case((3, 2, 2), 5, bc=("N",) * 6)
    try:
        se = c.se
        one = c.torch.ones(c.info.L, dtype=c.torch.float64, device=c.dev)
        y = c.empty()
        se.se_ax(c.m, one, y, se.SE_AX_ASSEMBLE)
        assert float(y.abs().max()) < 1e-12
        u, v = c.to_gpu(c.random_continuous(2, masked=False)), c.to_gpu(c.random_continuous(3, masked=False))
        au, av = c.empty(), c.empty()
        se.se_ax(c.m, u, au, se.SE_AX_ASSEMBLE)
        se.se_ax(c.m, v, av, se.SE_AX_ASSEMBLE)
        a, b = se.se_dot(c.m, v, au), se.se_dot(c.m, u, av)
        assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)
    finally:
        c.close()


@pytest.mark.parametrize("nel,p", SHAPES[::2])
def test_gs_dot_rhs_and_jacobi(nel, p):
    c = Case(nel, p, seed=20 + p)
    try:
        se = c.se
        u = wl.random_lvector(c.lv.gid.shape, 5)          # discontinuous L-vector
        g = c.to_gpu(u)
        se.se_gs(c.m, g, 1)
        assert rel_err(c.to_np(g), c.lv.mask * o.qqt(c.lv, u)) <= 1e-14
        g = c.to_gpu(u)
        se.se_gs(c.m, g, 0)
        assert rel_err(c.to_np(g), o.qqt(c.lv, u)) <= 1e-14
        a, b = c.random_continuous(6), c.random_continuous(7)
        d = se.se_dot(c.m, c.to_gpu(a), c.to_gpu(b))
        assert abs(d - o.dot(c.lv, a, b)) <= 1e-13 * max(1.0, abs(d))
        f = wl.f_rhs(*c.lv.X)
        bb = c.empty()
        se.se_mesh_rhs(c.m, c.to_gpu(f), bb)
        assert rel_err(c.to_np(bb), o.rhs(c.lv, f)) <= 1e-13
        dg = c.empty()
        se.se_jacobi_diag(c.m, dg)
        err = rel_err(c.to_np(dg), o.jacobi_diag(c.lv))
        assert err <= 1e-12, err
    finally:
        c.close()


def test_bounded_wait_returns_timeout_status():
    c = Case((1, 1, 1), 1)
    try:
        rc = c.se.se_selftest_wait_timeout(50.0)
        assert rc == c.se.SE_ETIMEOUT
        # the context is still usable afterwards
        y = c.empty()
        c.se.se_ax(c.m, c.to_gpu(np.ones(c.info.L)), y, 0)
        c.torch.cuda.synchronize()
    finally:
        c.close()


def test_invalid_arguments_are_rejected():
    _, se = Case((1, 1, 1), 1).torch, Case((1, 1, 1), 1).se
    with pytest.raises(se.SeError) as e:
        se.se_mesh_create((2, 2, 2), 11)
    assert e.value.code == se.SE_EINVAL
    with pytest.raises(se.SeError):
        se.se_mesh_create((0, 2, 2), 3)
    c = Case((2, 2, 2), 3)
    try:
        with pytest.raises(se.SeError):
            se.se_pmg_setup(c.m, se.pmg_desc((5, 3, 1)))          # schedule[0] != p
        with pytest.raises(se.SeError):
            se.se_pmg_setup(c.m, se.pmg_desc((3, 2)))             # coarsest must be p = 1
    finally:
        c.close()


def test_fp32_pipelined_operator_steady_state_and_residual_forms():
    """The persistent FP32 operator at p = 7 on a mesh large enough that every block loops over
    at least three element groups (so the stage refills and the mbarrier phase flips run), with a
    ragged last group (4095 elements is not a multiple of the group size), in its plain and its
    fused-residual forms, against the oracle element by element.  The residual form is reached
    through se_residual: r = M (b - QQ^T A_L u), the step r = b - A x of Algorithm 1.  The FP64
    (even-odd folded) and df64 residual forms are checked on the same mesh."""
    nel, p = (13, 15, 21), 7
    c = Case(nel, p, seed=41)
    try:
        se = c.se
        sms = c.torch.cuda.get_device_properties(0).multi_processor_count
        groups = -(-c.info.E // 4)                     # default group of 4 elements at p = 7
        assert groups >= 3 * sms and c.info.E % 4 != 0
        u = c.random_continuous(4, masked=False)
        ug, y = c.to_gpu(u), c.empty()
        se.se_ax(c.m, ug, y, se.SE_AX_FP32)
        assert rel_err(c.to_np(y), o.ax_local(c.lv, u)) <= 2e-5
        se.se_ax(c.m, ug, y, se.SE_AX_FP32 | se.SE_AX_ASSEMBLE)
        assert rel_err(c.to_np(y), o.ax(c.lv, u, mask=False)) <= 2e-5
        um = c.random_continuous(5)
        b = c.random_continuous(6)
        ref = b - o.ax(c.lv, um)
        r = c.empty()
        for flags, tol in ((se.SE_AX_FP32, 2e-5), (0, 1e-12), (se.SE_AX_DF64, 1e-12)):
            r.fill_(float("nan"))
            se.se_residual(c.m, c.to_gpu(b), c.to_gpu(um), r, flags)
            assert rel_err(c.to_np(r), ref) <= tol, flags
        with pytest.raises(se.SeError):
            se.se_residual(c.m, c.to_gpu(b), ug, ug, 0)
    finally:
        c.close()


@pytest.mark.parametrize("nel,p,bc", [
    ((13, 5, 4), 7, ("D",) * 6),                       # rows wrap inside blocks of 4 elements
    ((9, 4, 3), 5, ("D", "N", "N", "D", "D", "N")),    # blocks of 8, rows of 9
    ((8, 3, 5), 3, ("N", "D", "D", "N", "N", "D")),    # blocks of 8 aligned with rows
    ((1, 4, 6), 7, ("D",) * 6),                        # no x-interface
    ((21, 2, 2), 1, ("D", "D", "N", "N", "D", "D")),   # p = 1: blocks of 64 elements
    ((7, 6, 5), 9, ("D",) * 6),                        # blocks of 3
    ((16, 3, 2), 7, ("D", "N", "D", "D", "N", "D")),   # 4 blocks of 4 per row
    ((32, 2, 2), 5, ("N", "D", "D", "D", "D", "N")),   # 4 blocks of 8 per row
])
@pytest.mark.parametrize("fp32", [False, True])
def test_folded_operator_against_the_oracle(nel, p, bc, fp32):
    """The FP64 operator at even N and the FP32 pipelined operator do the x part of QQ^T and the
    Dirichlet mask inside their blocks (element groups), then the x-interfaces between blocks and
    the y and z directions: r = b - A u through se_residual on ragged and mixed-boundary meshes,
    element by element against the oracle (1e-12 in FP64, 2e-5 in FP32); all copies of every
    node bitwise equal."""
    c = Case(nel, p, seed=17, bc=bc)
    try:
        um = c.random_continuous(21)
        b = c.random_continuous(22)
        ref = b - o.ax(c.lv, um)
        r = c.empty()
        r.fill_(float("nan"))
        c.se.se_residual(c.m, c.to_gpu(b), c.to_gpu(um), r, c.se.SE_AX_FP32 if fp32 else 0)
        got = c.to_np(r)
        assert rel_err(got, ref) <= (2e-5 if fp32 else 1e-12)
        # copies of one node hold the same bits: scatter to global ids and back
        gid = c.lv.gid.reshape(-1)
        first = np.full(c.lv.n_global, -1, dtype=np.int64)
        first[gid[::-1]] = np.arange(gid.size)[::-1]
        flat = got.reshape(-1)
        assert np.array_equal(flat, flat[first[gid]])
    finally:
        c.close()
