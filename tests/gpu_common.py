"""Shared set-up for the GPU parity tests: builds the same mesh on both sides from the seeded
vertex lattice of workloads.py."""
import numpy as np
import pytest

import oracle as o
import workloads as wl

BC = {"D": 0, "N": 1}


def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_07663_gb300 import se
    return torch, se


class Case:
    """A mesh on the GPU (through the C ABI) and the same mesh in the oracle."""

    def __init__(self, nel, p, pert=0.05, seed=0, bc=("D",) * 6, amp=wl.DEFORM_AMP, V=None,
                 flags=0):
        self.torch, self.se = gpu()
        self.nel, self.p, self.bc, self.amp = tuple(nel), p, tuple(bc), amp
        self.V = wl.vertex_lattice(nel, pert, seed) if V is None else V
        self.m = self.se.se_mesh_create(nel, p, vertex_xyz=self.V, deform_amp=amp,
                                        bc=[BC[c] for c in bc], flags=flags)
        self.info = self.se.se_mesh_get_info(self.m)
        self.lv = o.make_level(self.V, nel, p, bc, amp)
        self.dev = self.torch.device("cuda:0")

    def to_gpu(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(self.dev)

    def to_np(self, t, shape=None):
        a = t.detach().cpu().numpy()
        return a.reshape(shape if shape is not None else self.lv.gid.shape)

    def empty(self, n=None):
        return self.torch.empty(n if n is not None else self.info.L, dtype=self.torch.float64,
                                device=self.dev)

    def random_continuous(self, seed, lv=None, masked=True):
        lv = lv or self.lv
        g = wl.random_lvector(lv.n_global, seed)
        u = o.from_global(lv, g)
        return lv.mask * u if masked else u

    def close(self):
        self.se.se_mesh_destroy(self.m)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
