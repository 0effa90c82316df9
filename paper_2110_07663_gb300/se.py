"""Thin ctypes binding of libse.so (include/se.h), argument marshalling only.

Every function keeps its C name.  Device vectors are passed as torch CUDA tensors (float64,
contiguous) or raw device pointers (int); streams as torch.cuda.Stream, raw handles or None.
A non-zero status raises SeError carrying the code and se_last_error().  The library must have
been built (``__graft_entry__.build()``); importing this module without it fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libse.so")

SE_OK, SE_EINVAL, SE_ENOMEM, SE_ENOTCONV, SE_ECUDA, SE_ETIMEOUT, SE_EBUSY, SE_EREFUSED, SE_ECANCELED = range(9)
SE_BC_DIRICHLET, SE_BC_NEUMANN = 0, 1
SE_FP64, SE_FP32, SE_DF64 = 0, 1, 2
SE_SMOOTH_JACOBI, SE_SMOOTH_RAS, SE_SMOOTH_ASM = 0, 1, 2
SE_CYCLE_MULTIPLICATIVE, SE_CYCLE_ADDITIVE = 0, 1
SE_FPCG, SE_FGMRES = 0, 1
SE_TOL_R0, SE_TOL_B = 0, 1
SE_AX_ASSEMBLE, SE_AX_MASK, SE_AX_FP32, SE_AX_DF64 = 1, 2, 4, 8
SE_MESH_NONBLOCKING_STREAM, SE_MESH_GS_MAP = 1, 2
SE_RHS_MODES, SE_RHS_HOST = 0, 1
SE_MAX_LEVELS, SE_MAX_ORDER = 8, 10
(SE_K_AX, SE_K_GS, SE_K_FDM, SE_K_CHEBY_UPD, SE_K_RESTRICT, SE_K_PROLONG, SE_K_COARSE,
 SE_K_KRYLOV, SE_K_JACOBI, SE_K_COUNT) = range(10)
KERNEL_NAMES = ["ax", "gs", "fdm", "cheby_update", "restrict", "prolong", "coarse_pcg", "krylov",
                "jacobi"]

STATUS_NAMES = {0: "SE_OK", 1: "SE_EINVAL", 2: "SE_ENOMEM", 3: "SE_ENOTCONV", 4: "SE_ECUDA",
                5: "SE_ETIMEOUT", 6: "SE_EBUSY", 7: "SE_EREFUSED", 8: "SE_ECANCELED"}


class SeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class se_mesh_desc(C.Structure):
    _fields_ = [("nel", C.c_int * 3), ("p", C.c_int), ("vertex_xyz", C.POINTER(C.c_double)),
                ("deform_amp", C.c_double), ("perturb_frac", C.c_double), ("seed", C.c_uint64),
                ("bc", C.c_int * 6), ("flags", C.c_int)]


class se_mesh_info(C.Structure):
    _fields_ = [("E", C.c_int64), ("N", C.c_int64), ("L", C.c_int64), ("n_global", C.c_int64),
                ("n_dof", C.c_int64), ("p", C.c_int), ("nel", C.c_int * 3)]


class se_pmg_desc(C.Structure):
    _fields_ = [("nlev", C.c_int), ("schedule", C.c_int * SE_MAX_LEVELS), ("smoother", C.c_int),
                ("cheb_order", C.c_int * SE_MAX_LEVELS), ("eig_lo", C.c_double),
                ("eig_hi", C.c_double), ("arnoldi_steps", C.c_int), ("seed", C.c_uint64),
                ("coarse_tol", C.c_double), ("coarse_maxit", C.c_int), ("precision", C.c_int),
                ("arnoldi_df64", C.c_int), ("cycle", C.c_int)]


class se_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("restart", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("graph_capture", C.c_int), ("stream", C.c_void_p),
                ("tol_norm", C.c_int), ("operator_df64", C.c_int)]


class se_problem(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("pmg", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p)]


class se_tile_cfg(C.Structure):
    _fields_ = [("p", C.c_int), ("precision", C.c_int), ("ax_elems_per_block", C.c_int),
                ("fdm_elems_per_block", C.c_int), ("ax_ms", C.c_double), ("fdm_ms", C.c_double)]


class se_request(C.Structure):
    _fields_ = [("mesh", se_mesh_desc), ("mesh_key", C.c_uint64), ("pmg", se_pmg_desc),
                ("rhs_kind", C.c_int), ("modes", C.c_int * 3), ("amplitude", C.c_double),
                ("b_host", C.POINTER(C.c_double)), ("x_host", C.POINTER(C.c_double)),
                ("tol", C.c_double), ("maxit", C.c_int)]


class se_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("rel_residual", C.c_double),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double), ("new_mesh", C.c_int),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


class se_serve_cfg(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int), ("builders", C.c_int),
                ("proj_vectors", C.c_int), ("operator_df64", C.c_int)]


class se_serve_summary(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("refused", C.c_int64),
                ("failed", C.c_int64), ("pending", C.c_int64), ("solves_per_s", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_concurrent", C.c_int), ("meshes_created", C.c_int64),
                ("mesh_reuses", C.c_int64), ("evictions", C.c_int64), ("resident_bytes", C.c_size_t),
                ("projected", C.c_int64), ("cancelled", C.c_int64)]


class se_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("rel_residual", C.c_double),
                ("ms_total", C.c_double), ("ms_precond", C.c_double), ("ms_operator", C.c_double)]


class se_tune_candidate(C.Structure):
    _fields_ = [("pmg", se_pmg_desc), ("setup_ms", C.c_double), ("ms", C.c_double),
                ("iterations", C.c_int), ("status", C.c_int)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libse.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
lib = C.CDLL(LIB_PATH)

_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
_SIGS = {
    "se_last_error": ([], C.c_char_p),
    "se_version": ([], C.c_int),
    "se_mesh_create": ([C.POINTER(se_mesh_desc), C.POINTER(_vp)], C.c_int),
    "se_mesh_destroy": ([_vp], C.c_int),
    "se_mesh_get_info": ([_vp, C.POINTER(se_mesh_info)], C.c_int),
    "se_mesh_nodes": ([_vp, _vp, _vp], C.c_int),
    "se_mesh_vertices": ([_vp, _dp], C.c_int),
    "se_mesh_rhs": ([_vp, _vp, _vp, _vp], C.c_int),
    "se_ax": ([_vp, _vp, _vp, _ip, _vp], C.c_int),
    "se_residual": ([_vp, _vp, _vp, _vp, _ip, _vp], C.c_int),
    "se_prof_fma_peak": ([_ip, C.POINTER(C.c_double), C.POINTER(_ip), _vp], C.c_int),
    "se_pmg_coarse_stats": ([_vp, _ip, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "se_gs": ([_vp, _vp, _ip, _vp], C.c_int),
    "se_gsmap_create": ([C.c_int64, _vp, _vp, C.POINTER(_vp)], C.c_int),
    "se_gsmap_apply": ([_vp, _vp, _ip, _vp], C.c_int),
    "se_gsmap_apply_f32": ([_vp, _vp, _ip, _vp], C.c_int),
    "se_gsmap_info": ([_vp, C.POINTER(C.c_int64)], C.c_int),
    "se_gsmap_count": ([C.c_int64, _vp, _vp, C.POINTER(C.c_int64)], C.c_int),
    "se_gsmap_destroy": ([_vp], C.c_int),
    "se_dot": ([_vp, _vp, _vp, _dp, _vp], C.c_int),
    "se_jacobi_diag": ([_vp, _vp, _vp], C.c_int),
    "se_pmg_setup": ([_vp, C.POINTER(se_pmg_desc), C.POINTER(_vp)], C.c_int),
    "se_pmg_destroy": ([_vp], C.c_int),
    "se_pmg_apply": ([_vp, _vp, _vp, _vp], C.c_int),
    "se_pmg_lambda": ([_vp, _ip, _dp], C.c_int),
    "se_pmg_level_info": ([_vp, _ip, C.POINTER(se_mesh_info)], C.c_int),
    "se_pmg_level_ax": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_smooth": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_gather_ext": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_fdm": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_cheby": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_restrict": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_prolong": ([_vp, _ip, _vp, _vp, _vp], C.c_int),
    "se_pmg_coarse_solve": ([_vp, _vp, _vp, C.POINTER(C.c_int), _vp], C.c_int),
    "se_pmg_coarse_solve_noalloc": ([_vp, _vp, _vp, C.POINTER(C.c_int), _vp], C.c_int),
    "se_solve": ([_vp, _vp, _vp, _vp, C.POINTER(se_solve_opts), C.POINTER(se_solve_stats)], C.c_int),
    "se_solve_host": ([_vp, _vp, _vp, _vp, _vp, C.POINTER(se_solve_opts), C.POINTER(se_solve_stats)],
                      C.c_int),
    "se_batch_create": ([_ip, C.POINTER(se_problem), C.POINTER(se_solve_opts), C.POINTER(_vp)], C.c_int),
    "se_batch_run": ([_vp, _vp], C.c_int),
    "se_batch_stats": ([_vp, _vp, C.POINTER(se_solve_stats)], C.c_int),
    "se_batch_destroy": ([_vp], C.c_int),
    "se_batch_solve": ([_ip, C.POINTER(se_problem), C.POINTER(se_solve_opts), C.POINTER(se_solve_stats)], C.c_int),
    "se_batch_info": ([_vp, C.POINTER(_ip), C.POINTER(_ip)], C.c_int),
    "se_tune": ([_ip, _ip, C.POINTER(se_tile_cfg)], C.c_int),
    "se_tune_get": ([_ip, _ip, C.POINTER(se_tile_cfg)], C.c_int),
    "se_tune_set": ([C.POINTER(se_tile_cfg)], C.c_int),
    "se_pmg_autotune_space": ([_ip, _ip, C.POINTER(se_tune_candidate), _ip, C.POINTER(C.c_int)], C.c_int),
    "se_pmg_autotune": ([_vp, _vp, C.POINTER(se_solve_opts), _ip, C.POINTER(se_tune_candidate), _ip,
                         C.POINTER(C.c_int), C.POINTER(_vp)], C.c_int),
    "se_mesh_footprint_bytes": ([C.POINTER(se_mesh_desc), C.POINTER(se_pmg_desc), C.POINTER(C.c_size_t)], C.c_int),
    "se_proj_create": ([_vp, C.c_int, C.POINTER(_vp)], C.c_int),
    "se_proj_destroy": ([_vp], C.c_int),
    "se_proj_guess": ([_vp, _vp, _vp, _vp], C.c_int),
    "se_proj_update": ([_vp, _vp, C.POINTER(C.c_int), _vp], C.c_int),
    "se_serve_create": ([C.POINTER(se_serve_cfg), C.POINTER(_vp)], C.c_int),
    "se_serve_submit": ([_vp, C.POINTER(se_request), C.POINTER(C.c_uint64)], C.c_int),
    "se_serve_poll": ([_vp, C.c_uint64, C.POINTER(se_result)], C.c_int),
    "se_serve_wait": ([_vp, C.c_uint64, C.c_double, C.POINTER(se_result)], C.c_int),
    "se_serve_stats": ([_vp, C.POINTER(se_serve_summary)], C.c_int),
    "se_serve_cancel": ([_vp, C.c_uint64], C.c_int),
    "se_serve_destroy": ([_vp], C.c_int),
    "se_prof_enable": ([_ip], C.c_int),
    "se_prof_reset": ([], C.c_int),
    "se_prof_query": ([_ip, _dp, C.POINTER(C.c_int64), _dp, _dp, _dp], C.c_int),
    "se_prof_query_variant": ([_ip, _ip, _dp, C.POINTER(C.c_int64), _dp, _dp, _dp], C.c_int),
    "se_selftest_wait_timeout": ([C.c_double], C.c_int),
    "se_selftest_fail_alloc": ([C.c_int], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


def se_last_error() -> str:
    return lib.se_last_error().decode()


def _check(code: int, allow=()):
    if code != SE_OK and code not in allow:
        raise SeError(code, se_last_error())
    return code


def _ptr(x):
    """Device pointer of a contiguous CUDA tensor (or a raw int pointer)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ----------------------------------------------------------------------------- mesh / operator
def se_mesh_create(nel, p, *, vertex_xyz=None, deform_amp=0.05, perturb_frac=0.0, seed=0,
                   bc=(SE_BC_DIRICHLET,) * 6, flags=0):
    """Create a mesh; vertex_xyz is an optional host float64 array of shape (V, 3)."""
    d = se_mesh_desc()
    d.nel[:] = list(nel)
    d.p = p
    keep = None
    if vertex_xyz is not None:
        import numpy as np
        keep = np.ascontiguousarray(vertex_xyz, dtype=np.float64).reshape(-1)
        d.vertex_xyz = keep.ctypes.data_as(C.POINTER(C.c_double))
    d.deform_amp = deform_amp
    d.perturb_frac = perturb_frac
    d.seed = seed
    d.bc[:] = list(bc)
    d.flags = flags
    h = _vp()
    _check(lib.se_mesh_create(C.byref(d), C.byref(h)))
    return h.value


def se_mesh_destroy(m):
    _check(lib.se_mesh_destroy(m))


def se_mesh_get_info(m) -> se_mesh_info:
    info = se_mesh_info()
    _check(lib.se_mesh_get_info(m, C.byref(info)))
    return info


def se_mesh_nodes(m, xyz, stream=None):
    _check(lib.se_mesh_nodes(m, _ptr(xyz), _stream(stream)))


def se_mesh_vertices(m, out_np):
    _check(lib.se_mesh_vertices(m, out_np.ctypes.data_as(C.POINTER(C.c_double))))


def se_mesh_rhs(m, f, b, stream=None):
    _check(lib.se_mesh_rhs(m, _ptr(f), _ptr(b), _stream(stream)))


def se_ax(m, u, y, flags=SE_AX_ASSEMBLE | SE_AX_MASK, stream=None):
    _check(lib.se_ax(m, _ptr(u), _ptr(y), flags, _stream(stream)))


def se_residual(m, b, u, r, flags=0, stream=None):
    _check(lib.se_residual(m, _ptr(b), _ptr(u), _ptr(r), flags, _stream(stream)))


def se_gs(m, u, mask=1, stream=None):
    _check(lib.se_gs(m, _ptr(u), mask, _stream(stream)))


# ----------------------------------------------------------------------------- QQ^T index map
def _gsmap_host_args(gid, dirichlet):
    import numpy as np
    g = np.ascontiguousarray(gid, dtype=np.int64).reshape(-1)
    d = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
    if d is not None and d.size != g.size:
        raise ValueError("dirichlet must have one byte per local point")
    return g, d, g.ctypes.data, (None if d is None else d.ctypes.data)


def se_gsmap_create(gid, dirichlet=None):
    """Index-map QQ^T for the global ids `gid` (host array, one per local point)."""
    g, d, gp, dp = _gsmap_host_args(gid, dirichlet)
    h = _vp()
    _check(lib.se_gsmap_create(g.size, gp, dp, C.byref(h)))
    return h.value


def se_gsmap_apply(g, u, mask=1, stream=None):
    """In place u <- [M] QQ^T u; u is a float64 or float32 CUDA tensor."""
    import torch
    fn = lib.se_gsmap_apply_f32 if u.dtype == torch.float32 else lib.se_gsmap_apply
    _check(fn(g, _ptr(u), mask, _stream(stream)))


def se_gsmap_info(g):
    c = (C.c_int64 * 5)()
    _check(lib.se_gsmap_info(g, c))
    return tuple(c)


def se_gsmap_count(gid, dirichlet=None):
    """Bucket counts (pairs, quads, octets, other groups, masked singles); host only."""
    g, d, gp, dp = _gsmap_host_args(gid, dirichlet)
    c = (C.c_int64 * 5)()
    _check(lib.se_gsmap_count(g.size, gp, dp, c))
    return tuple(c)


def se_gsmap_destroy(g):
    _check(lib.se_gsmap_destroy(g))


def se_dot(m, a, b, stream=None) -> float:
    out = C.c_double()
    _check(lib.se_dot(m, _ptr(a), _ptr(b), C.byref(out), _stream(stream)))
    return out.value


def se_jacobi_diag(m, d, stream=None):
    _check(lib.se_jacobi_diag(m, _ptr(d), _stream(stream)))


# ----------------------------------------------------------------------------- p-multigrid
def pmg_desc(schedule, smoother=SE_SMOOTH_RAS, cheb_order=2, eig_lo=0.1, eig_hi=1.1,
             arnoldi_steps=10, seed=0, coarse_tol=1e-2, coarse_maxit=500, precision=SE_FP64,
             arnoldi_df64=0, cycle=SE_CYCLE_MULTIPLICATIVE):
    d = se_pmg_desc()
    d.nlev = len(schedule)
    d.schedule[:len(schedule)] = list(schedule)
    d.smoother = smoother
    orders = cheb_order if isinstance(cheb_order, (list, tuple)) else [cheb_order] * len(schedule)
    d.cheb_order[:len(orders)] = list(orders)
    d.eig_lo, d.eig_hi = eig_lo, eig_hi
    d.arnoldi_steps = arnoldi_steps
    d.seed = seed
    d.coarse_tol, d.coarse_maxit = coarse_tol, coarse_maxit
    d.precision = precision
    d.arnoldi_df64 = arnoldi_df64
    d.cycle = cycle
    return d


def se_pmg_setup(m, desc: se_pmg_desc):
    h = _vp()
    _check(lib.se_pmg_setup(m, C.byref(desc), C.byref(h)))
    return h.value


def se_pmg_destroy(P):
    _check(lib.se_pmg_destroy(P))


def se_pmg_apply(P, r, z, stream=None):
    _check(lib.se_pmg_apply(P, _ptr(r), _ptr(z), _stream(stream)))


def se_pmg_lambda(P, lvl) -> float:
    out = C.c_double()
    _check(lib.se_pmg_lambda(P, lvl, C.byref(out)))
    return out.value


def se_pmg_level_info(P, lvl) -> se_mesh_info:
    info = se_mesh_info()
    _check(lib.se_pmg_level_info(P, lvl, C.byref(info)))
    return info


def _lvl_call(fn):
    def call(P, lvl, a, b, stream=None):
        _check(fn(P, lvl, _ptr(a), _ptr(b), _stream(stream)))
    return call


se_pmg_level_ax = _lvl_call(lib.se_pmg_level_ax)
se_pmg_smooth = _lvl_call(lib.se_pmg_smooth)
se_pmg_gather_ext = _lvl_call(lib.se_pmg_gather_ext)
se_pmg_fdm = _lvl_call(lib.se_pmg_fdm)
se_pmg_cheby = _lvl_call(lib.se_pmg_cheby)
se_pmg_restrict = _lvl_call(lib.se_pmg_restrict)
se_pmg_prolong = _lvl_call(lib.se_pmg_prolong)


def se_pmg_coarse_solve(P, r, x, stream=None) -> int:
    it = C.c_int()
    _check(lib.se_pmg_coarse_solve(P, _ptr(r), _ptr(x), C.byref(it), _stream(stream)))
    return it.value


def se_pmg_coarse_stats(P, reset=False):
    """(coarse solves, total coarse Jacobi-PCG iterations) since the last reset."""
    n, it = C.c_int64(), C.c_int64()
    _check(lib.se_pmg_coarse_stats(P, 1 if reset else 0, C.byref(n), C.byref(it)))
    return n.value, it.value


def se_pmg_coarse_solve_noalloc(P, r, x, stream=None) -> int:
    """Coarse solve whose work space is the library's static device array (no allocation)."""
    it = C.c_int()
    _check(lib.se_pmg_coarse_solve_noalloc(P, _ptr(r), _ptr(x), C.byref(it), _stream(stream)))
    return it.value


# ----------------------------------------------------------------------------- solve
def se_solve(m, P, b, x, method=SE_FPCG, tol=1e-8, maxit=1000, restart=20, graph_capture=0,
             stream=None, allow_notconv=False, tol_norm=0, operator_df64=0) -> se_solve_stats:
    o = se_solve_opts()
    o.method, o.restart, o.tol, o.maxit, o.graph_capture = method, restart, tol, maxit, graph_capture
    o.tol_norm = tol_norm
    o.operator_df64 = operator_df64
    o.stream = _stream(stream)
    st = se_solve_stats()
    _check(lib.se_solve(m, P, _ptr(b), _ptr(x), C.byref(o), C.byref(st)),
           allow=(SE_ENOTCONV,) if allow_notconv else ())
    return st


def _host_ptr(a):
    """Address of a contiguous float64 host array (CPU tensor or numpy array); None -> NULL."""
    if a is None:
        return None
    if hasattr(a, "is_cuda"):
        if a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous():
            raise ValueError("expected a contiguous float64 CPU tensor")
        return a.data_ptr()
    if a.dtype.itemsize != 8 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous float64 array")
    return a.ctypes.data


def se_solve_host(m, P, b_host, x_host, x0_host=None, method=SE_FPCG, tol=1e-8, maxit=1000,
                  restart=20, graph_capture=0, stream=None, allow_notconv=False, tol_norm=0,
                  operator_df64=0) -> se_solve_stats:
    """se_solve with host buffers (the copies inside the library call); x starts from zero unless
    x0_host is given."""
    o = se_solve_opts()
    o.method, o.restart, o.tol, o.maxit, o.graph_capture = method, restart, tol, maxit, graph_capture
    o.tol_norm = tol_norm
    o.operator_df64 = operator_df64
    o.stream = _stream(stream)
    st = se_solve_stats()
    _check(lib.se_solve_host(m, P, _host_ptr(b_host), _host_ptr(x0_host), _host_ptr(x_host), C.byref(o),
                             C.byref(st)),
           allow=(SE_ENOTCONV,) if allow_notconv else ())
    return st


# ----------------------------------------------------------------------------- preconditioner autotuner
def se_pmg_autotune_space(p, precision=SE_FP64):
    """The default candidate space for order p (Sec. 5, Table 5 without SEMFEM)."""
    arr = (se_tune_candidate * 8)()
    n = C.c_int()
    _check(lib.se_pmg_autotune_space(int(p), int(precision), arr, 8, C.byref(n)))
    return [arr[i] for i in range(n.value)]


def se_pmg_autotune(m, b, candidates, repeats=2, method=SE_FPCG, tol=1e-8, maxit=1000, restart=20,
                    graph_capture=1, tol_norm=0, keep=True, operator_df64=0):
    """Times every candidate; returns (best index, timed candidates, best preconditioner or None)."""
    o = se_solve_opts()
    o.method, o.restart, o.tol, o.maxit, o.graph_capture = method, restart, tol, maxit, graph_capture
    o.tol_norm = tol_norm
    o.operator_df64 = operator_df64
    arr = (se_tune_candidate * len(candidates))(*candidates)
    best = C.c_int(-1)
    h = _vp()
    _check(lib.se_pmg_autotune(m, _ptr(b), C.byref(o), int(repeats), arr, len(candidates),
                               C.byref(best), C.byref(h) if keep else None))
    return best.value, [arr[i] for i in range(len(candidates))], h.value if keep else None


# ----------------------------------------------------------------------------- projection
def se_proj_create(m, max_vectors=10):
    h = _vp()
    _check(lib.se_proj_create(m, int(max_vectors), C.byref(h)))
    return h.value


def se_proj_destroy(p):
    _check(lib.se_proj_destroy(p))


def se_proj_guess(p, b, x, stream=None):
    _check(lib.se_proj_guess(p, _ptr(b), _ptr(x), _stream(stream)))


def se_proj_update(p, x, stream=None) -> int:
    n = C.c_int()
    _check(lib.se_proj_update(p, _ptr(x), C.byref(n), _stream(stream)))
    return n.value


# ----------------------------------------------------------------------------- batched solves
def _problems(problems):
    arr = (se_problem * len(problems))()
    for i, (m, P, b, x) in enumerate(problems):
        arr[i].mesh, arr[i].pmg, arr[i].b, arr[i].x = m, P, _ptr(b), _ptr(x)
    return arr


def _opts(tol, maxit, stream, method=SE_FPCG, restart=20, graph_capture=1, tol_norm=0):
    o = se_solve_opts()
    o.method, o.restart, o.tol, o.maxit, o.graph_capture = method, restart, tol, maxit, graph_capture
    o.tol_norm = tol_norm
    o.stream = _stream(stream)
    return o


def se_batch_create(problems, tol=1e-8, maxit=1000, stream=None, operator_df64=0, tol_norm=0,
                    graph_capture=1):
    """problems: list of (mesh, pmg or None, b, x).  Returns the batch handle."""
    arr = _problems(problems)
    h = _vp()
    o = _opts(tol, maxit, stream, tol_norm=tol_norm, graph_capture=graph_capture)
    o.operator_df64 = operator_df64
    _check(lib.se_batch_create(len(problems), arr, C.byref(o), C.byref(h)))
    return h.value


def se_batch_run(B, stream=None):
    _check(lib.se_batch_run(B, _stream(stream)))


def se_batch_stats(B, n, stream=None, allow_notconv=False):
    out = (se_solve_stats * n)()
    _check(lib.se_batch_stats(B, _stream(stream), out), allow=(SE_ENOTCONV,) if allow_notconv else ())
    return list(out)


def se_batch_info(B):
    """(groups, problems in groups) of a batch."""
    g, k = _ip(), _ip()
    _check(lib.se_batch_info(B, C.byref(g), C.byref(k)))
    return g.value, k.value


def se_batch_destroy(B):
    _check(lib.se_batch_destroy(B))


def se_batch_solve(problems, tol=1e-8, maxit=1000, stream=None, allow_notconv=False, tol_norm=0):
    arr = _problems(problems)
    out = (se_solve_stats * len(problems))()
    _check(lib.se_batch_solve(len(problems), arr, C.byref(_opts(tol, maxit, stream, tol_norm=tol_norm)), out),
           allow=(SE_ENOTCONV,) if allow_notconv else ())
    return list(out)


# ----------------------------------------------------------------------------- tile autotuner
def se_tune(p, precision=SE_FP64) -> se_tile_cfg:
    out = se_tile_cfg()
    _check(lib.se_tune(p, precision, C.byref(out)))
    return out


def se_tune_get(p, precision=SE_FP64) -> se_tile_cfg:
    out = se_tile_cfg()
    _check(lib.se_tune_get(p, precision, C.byref(out)))
    return out


def se_tune_set(p, precision, ax_elems_per_block, fdm_elems_per_block):
    c = se_tile_cfg()
    c.p, c.precision = p, precision
    c.ax_elems_per_block, c.fdm_elems_per_block = ax_elems_per_block, fdm_elems_per_block
    _check(lib.se_tune_set(C.byref(c)))


# ----------------------------------------------------------------------------- serving
def mesh_desc(nel, p, perturb_frac=0.0, seed=0, deform_amp=0.05, bc=(SE_BC_DIRICHLET,) * 6, flags=0):
    d = se_mesh_desc()
    d.nel[:] = list(nel)
    d.p, d.deform_amp, d.perturb_frac, d.seed, d.flags = p, deform_amp, perturb_frac, seed, flags
    d.bc[:] = list(bc)
    return d


def se_mesh_footprint_bytes(mdesc: se_mesh_desc, pdesc: se_pmg_desc) -> int:
    out = C.c_size_t()
    _check(lib.se_mesh_footprint_bytes(C.byref(mdesc), C.byref(pdesc), C.byref(out)))
    return out.value


def make_request(mdesc, mesh_key, pdesc, modes=(1, 1, 1), amplitude=1.0, b_host=None,
                 x_host=None, tol=1e-8, maxit=500) -> se_request:
    """Request for se_serve_submit; b_host / x_host are numpy float64 arrays (kept alive by the
    caller until the request completes; b_host is copied at submission)."""
    q = se_request()
    q.mesh, q.mesh_key, q.pmg = mdesc, mesh_key, pdesc
    q.rhs_kind = SE_RHS_HOST if b_host is not None else SE_RHS_MODES
    q.modes[:] = list(modes)
    q.amplitude = amplitude
    if b_host is not None:
        q.b_host = b_host.ctypes.data_as(C.POINTER(C.c_double))
    if x_host is not None:
        q.x_host = x_host.ctypes.data_as(C.POINTER(C.c_double))
    q.tol, q.maxit = tol, maxit
    return q


def se_serve_create(hbm_budget, max_slots, builders=0, proj_vectors=0, operator_df64=0):
    c = se_serve_cfg()
    c.hbm_budget, c.max_slots, c.builders = int(hbm_budget), int(max_slots), int(builders)
    c.proj_vectors = int(proj_vectors)
    c.operator_df64 = int(operator_df64)
    h = _vp()
    _check(lib.se_serve_create(C.byref(c), C.byref(h)))
    return h.value


def se_serve_submit(S, req: se_request) -> int:
    t = C.c_uint64()
    _check(lib.se_serve_submit(S, C.byref(req), C.byref(t)))
    return t.value


def se_serve_poll(S, ticket):
    """(status, se_result) with status SE_EBUSY while pending."""
    r = se_result()
    rc = lib.se_serve_poll(S, ticket, C.byref(r))
    if rc not in (SE_OK, SE_EBUSY, SE_ENOTCONV, SE_ECANCELED):
        raise SeError(rc, se_last_error())
    return rc, r


def se_serve_wait(S, ticket, timeout_ms=60000.0, allow=()):
    r = se_result()
    _check(lib.se_serve_wait(S, ticket, timeout_ms, C.byref(r)), allow=allow)
    return r


def se_serve_cancel(S, ticket) -> int:
    """SE_OK if the queued request was removed (its result: SE_ECANCELED), SE_EBUSY if it has
    started (it completes normally)."""
    return _check(lib.se_serve_cancel(S, ticket), allow=(SE_EBUSY,))


def se_serve_stats(S) -> se_serve_summary:
    out = se_serve_summary()
    _check(lib.se_serve_stats(S, C.byref(out)))
    return out


def se_serve_destroy(S):
    _check(lib.se_serve_destroy(S))


# ----------------------------------------------------------------------------- profiling
def se_prof_enable(on=True):
    _check(lib.se_prof_enable(1 if on else 0))


def se_prof_reset():
    _check(lib.se_prof_reset())


def se_prof_query(kind):
    ms, n, units, by, fl = C.c_double(), C.c_int64(), C.c_double(), C.c_double(), C.c_double()
    _check(lib.se_prof_query(kind, C.byref(ms), C.byref(n), C.byref(units), C.byref(by), C.byref(fl)))
    return dict(ms=ms.value, launches=n.value, units=units.value, bytes=by.value, flops=fl.value)


def se_prof_query_variant(kind, variant):
    ms, n, units, by, fl = C.c_double(), C.c_int64(), C.c_double(), C.c_double(), C.c_double()
    _check(lib.se_prof_query_variant(kind, variant, C.byref(ms), C.byref(n), C.byref(units),
                                     C.byref(by), C.byref(fl)))
    return dict(ms=ms.value, launches=n.value, units=units.value, bytes=by.value, flops=fl.value)


def se_selftest_wait_timeout(timeout_ms=100.0) -> int:
    return lib.se_selftest_wait_timeout(timeout_ms)


def se_prof_fma_peak(kind, stream=None):
    """Measured FMA throughput (TFLOP/s) and SM count: kind 0 FP64, 1 FP32, 2 packed FP32 pairs."""
    t, n = C.c_double(), _ip()
    _check(lib.se_prof_fma_peak(int(kind), C.byref(t), C.byref(n), _stream(stream)))
    return t.value, n.value


def se_selftest_fail_alloc(n):
    """Arm (n >= 1) or disarm (0) the injected failure of the n-th following device allocation."""
    _check(lib.se_selftest_fail_alloc(int(n)))
