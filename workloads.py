"""Seeded synthetic inputs shared by the oracle, the tests and bench.py.

This module holds no arithmetic of the solver: it only defines the synthetic workloads (mesh
vertex lattices, right-hand-side functions, random vectors, request streams) and the one
counter-based generator that both sides draw from.

Counter-based generator: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the constants of Vigna's public-domain
splitmix64.c).  Value number ``c`` of stream ``seed`` is ``mix(seed + (c + 1) * GOLDEN)``; the
uniform double is the top 53 bits times 2^-53.  The CUDA library implements the same published
definition independently in C++ for the random draws it makes itself (vertex perturbation when no
vertex array is supplied, Arnoldi start vectors).

Workloads stand in for the paper's Kershaw and Navier-Stokes meshes, whose map formula and mesh
files are not available: a box [0,1]^3 split into nx*ny*nz hexahedra, interior lattice vertices
moved by a seeded uniform perturbation of at most ``perturb_frac`` of the element width, and the
smooth map x_c <- x_c + amp*sin(2 pi x)sin(2 pi y)sin(2 pi z) applied to every node.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """SplitMix64 output number ``counter`` (array) of stream ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % (1 << 64)) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of SplitMix64 times 2^-53."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def vertex_lattice(nel, perturb_frac: float = 0.0, seed: int = 0) -> np.ndarray:
    """Vertex lattice of the box [0,1]^3 split into nel=(nx,ny,nz) hexahedra.

    Returns V with shape (nz+1, ny+1, nx+1, 3); vertex (a,b,c) has id v = a + (nx+1)(b + (ny+1)c).
    Interior vertices move by perturb_frac*h_d*(2U-1) in each direction d, with U the uniform
    number 3v+d of stream ``seed``; vertices on the boundary stay fixed.
    """
    nx, ny, nz = nel
    a = np.arange(nx + 1) / nx
    b = np.arange(ny + 1) / ny
    c = np.arange(nz + 1) / nz
    V = np.empty((nz + 1, ny + 1, nx + 1, 3))
    V[..., 0] = a[None, None, :]
    V[..., 1] = b[None, :, None]
    V[..., 2] = c[:, None, None]
    if perturb_frac != 0.0:
        vid = np.arange((nx + 1) * (ny + 1) * (nz + 1), dtype=np.uint64).reshape(nz + 1, ny + 1, nx + 1)
        interior = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
        interior[1:nz, 1:ny, 1:nx] = True
        h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        for d in range(3):
            u = uniform01(seed, vid * np.uint64(3) + np.uint64(d))
            V[..., d] += np.where(interior, perturb_frac * h[d] * (2.0 * u - 1.0), 0.0)
    return V


def _zigzag(t, segments):
    """Piecewise-linear wave on [0,1]: +1 at t = 0, alternating -1/+1 at t = k/segments."""
    s = np.asarray(t) * segments
    k = np.clip(np.floor(s), 0, segments - 1)
    f = s - k
    sign = np.where(k % 2 == 0, 1.0, -1.0)
    return sign * (1.0 - 2.0 * f)


def _split_map(v, t):
    """Monotone piecewise-linear map of [0,1] onto itself sending 1/2 to t (0 < t < 1)."""
    return np.where(v <= 0.5, 2.0 * t * v, t + 2.0 * (1.0 - t) * (v - 0.5))


def skewed_lattice(nel, eps: float, segments: int = 2) -> np.ndarray:
    """A strongly skewed vertex lattice of [0,1]^3, a stand-in for the paper's Kershaw meshes
    (Sec. 3.1; the paper does not give their map): eps = 1 is the uniform box, smaller eps squeezes
    half of each column of elements and stretches the other half, with the split point moving
    along a zigzag in the other coordinates, so that elements are sheared and their aspect
    ratios reach (2 - eps)/eps and their shear dy/dx up to 2 segments (1 - eps) v.  With the
    default two pieces, eps = 0.3 converges in about 30 iterations of the paper's default
    preconditioner, the range the paper reports for its moderately skewed mesh (six pieces,
    shear up to 4.2, take about 200).

    x = a;  y = split(b, t1(a));  z = split(c, t2(a, b)), with split the monotone
    piecewise-linear map sending 1/2 to t, t1 = 1/2 + (1 - eps)/2 zigzag(a),
    t2 = 1/2 + (1 - eps)/2 zigzag(a) zigzag(b), and zigzag the +-1 wave with ``segments`` linear
    pieces.  Same layout as ``vertex_lattice``; the boundary faces stay on the unit cube.
    """
    assert 0.0 < eps <= 1.0
    nx, ny, nz = nel
    a = (np.arange(nx + 1) / nx)[None, None, :]
    b = (np.arange(ny + 1) / ny)[None, :, None]
    c = (np.arange(nz + 1) / nz)[:, None, None]
    amp = 0.5 * (1.0 - eps)
    t1 = 0.5 + amp * _zigzag(a, segments)
    t2 = 0.5 + amp * _zigzag(a, segments) * _zigzag(b, segments)
    V = np.empty((nz + 1, ny + 1, nx + 1, 3))
    V[..., 0] = np.broadcast_to(a, V.shape[:3])
    V[..., 1] = np.broadcast_to(_split_map(b, t1), V.shape[:3])
    V[..., 2] = np.broadcast_to(_split_map(c, t2), V.shape[:3])
    return V


def arnoldi_start_global(seed: int, n_global: int) -> np.ndarray:
    """Start vector of the Chebyshev bound estimate: 2U-1 per global node id (stream ``seed``)."""
    return 2.0 * uniform01(seed, np.arange(n_global, dtype=np.uint64)) - 1.0


def arnoldi_seed(pmg_seed: int, level: int) -> int:
    """Stream used for the start vector of level ``level`` (same rule on both sides)."""
    return 1000 + level + 7919 * pmg_seed


# Right-hand side of the manufactured problem u* = sin(pi x) sin(pi y) sin(pi z), -lap u* = f.
def u_exact(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def f_rhs(x, y, z):
    return 3.0 * np.pi ** 2 * u_exact(x, y, z)


def u_exact_modes(x, y, z, k, a):
    """u* = a * prod_c sin(k_c pi x_c), used for batched and served requests."""
    return a * np.sin(k[0] * np.pi * x) * np.sin(k[1] * np.pi * y) * np.sin(k[2] * np.pi * z)


def f_rhs_modes(x, y, z, k, a):
    return np.pi ** 2 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2) * u_exact_modes(x, y, z, k, a)


def request_modes(seed: int):
    """Per-request manufactured-solution parameters: k_c in {1,2,3}, amplitude in [0.5, 2)."""
    u = uniform01(seed, np.arange(4, dtype=np.uint64))
    k = tuple(int(1 + min(2, math.floor(3 * v))) for v in u[:3])
    return k, 0.5 + 1.5 * float(u[3])


def random_lvector(shape, seed: int) -> np.ndarray:
    """Seeded uniform[-1,1] array of the given shape (numpy PCG64)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


# ---------------------------------------------------------------------------------------------
# Workload definitions (synthetic stand-ins for the paper's meshes).
# ---------------------------------------------------------------------------------------------
DEFORM_AMP = 0.05

SMALL_BOX = dict(name="box4x4x4_p7", nel=(4, 4, 4), p=7, perturb_frac=0.0, seed=0,
                 schedule=(7, 3, 1), cheb_order=2)
LARGE_BOX = dict(name="box32x32x32_p7", nel=(32, 32, 32), p=7, perturb_frac=0.05, seed=0,
                 schedule=(7, 5, 3, 1), cheb_order=2)
PRECISION_P9_SCHEDULE = (9, 5, 1)
BATCH_ELEMENTS = (8, 12, 16, 20, 24)
BATCH_ORDERS = (3, 5, 7, 9)
BATCH_SCHEDULES = {3: (3, 1), 5: (5, 3, 1), 7: (7, 3, 1), 9: (9, 5, 1)}


def batch_problems(n: int = 64, seed0: int = 0):
    """n independent problems: E from {8^3..24^3} and p from {3,5,7,9}, drawn per seed."""
    out = []
    for s in range(seed0, seed0 + n):
        u = uniform01(50000 + s, np.arange(2, dtype=np.uint64))
        m = BATCH_ELEMENTS[int(u[0] * len(BATCH_ELEMENTS))]
        p = BATCH_ORDERS[int(u[1] * len(BATCH_ORDERS))]
        out.append(dict(nel=(m, m, m), p=p, perturb_frac=0.05, seed=s,
                        schedule=BATCH_SCHEDULES[p], modes=request_modes(s)))
    return out


def serve_requests(n: int = 10000, rate: float = 200.0, seed: int = 0, reuse_frac: float = 0.3,
                   orders=(5, 7, 9), emin: int = 512, emax: int = 65536, n_resident: int = 8):
    """Poisson arrival stream: E log-uniform in [emin, emax], p from ``orders``; a fraction
    ``reuse_frac`` of requests reuse one of the first ``n_resident`` distinct meshes."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    meshes = []
    for i in range(n):
        if meshes and rng.uniform() < reuse_frac:
            mesh = meshes[int(rng.integers(0, min(len(meshes), n_resident)))]
        else:
            E = math.exp(rng.uniform(math.log(emin), math.log(emax)))
            nx = max(1, round(E ** (1.0 / 3.0)))
            nz = max(1, round(E / (nx * nx)))
            p = int(orders[int(rng.integers(0, len(orders)))])
            mesh = dict(nel=(nx, nx, nz), p=p, perturb_frac=0.05, seed=int(rng.integers(0, 1 << 30)))
            meshes.append(mesh)
        reqs.append(dict(t=float(t[i]), mesh=mesh, rhs_seed=int(rng.integers(0, 1 << 30))))
    return reqs
