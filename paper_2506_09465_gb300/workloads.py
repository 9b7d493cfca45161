"""Seeded synthetic inputs for tests and the benchmark. Holds no step of the method: it only
builds grids, relaxation-time fields, wall temperatures, sources and band tables with the
shapes of the paper's workloads (arXiv 2506.09465 Sec. 4) and of the larger configurations
run here. Imported by tests, bench.py and __graft_entry__; never by oracle/ or the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Instance:
    dim: int
    n: tuple
    L: tuple
    tau: np.ndarray          # [nb, ncells]
    wall_T: np.ndarray       # [2*dim]
    source: Optional[np.ndarray] = None

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n[: self.dim]))


@dataclass
class Workload:
    name: str
    C: np.ndarray
    v: np.ndarray
    instances: List[Instance] = field(default_factory=list)
    particles_per_cell: int = 1024
    particles_per_wall_face: int = 1024

    @property
    def nb(self) -> int:
        return len(self.C)

    @property
    def total_cells(self) -> int:
        return sum(i.ncells for i in self.instances)


def slab(n=50, Kn=1.0, T_left=1.0, T_right=-1.0, particles=1000) -> Workload:
    """1D gray film (Sec. 4.1 shape): L = 1, C = |v| = 1, tau = Kn, black walls."""
    inst = Instance(1, (n,), (1.0,), np.full((1, n), Kn), np.array([T_left, T_right]))
    return Workload(f"1D gray slab {n} cells Kn={Kn}", np.array([1.0]), np.array([1.0]), [inst], particles, particles)


def cavity(n=128, Kn=1.0, particles=1024) -> Workload:
    """2D gray square cavity (Sec. 4.4 shape): unit square, top wall T = 1, others 0."""
    inst = Instance(2, (n, n), (1.0, 1.0), np.full((1, n * n), Kn), np.array([0.0, 0.0, 0.0, 1.0]))
    return Workload(f"2D gray cavity {n}x{n} Kn={Kn}", np.array([1.0]), np.array([1.0]), [inst], particles, particles)


def cavity_sweep(n=128, Kns=(0.01, 0.1, 1.0, 10.0), particles=1024) -> Workload:
    """The 2D cavity at several Knudsen numbers, one instance each (one batched context)."""
    insts = [Instance(2, (n, n), (1.0, 1.0), np.full((1, n * n), k), np.array([0.0, 0.0, 0.0, 1.0])) for k in Kns]
    return Workload(f"2D gray cavity {n}x{n} Kn={list(Kns)}", np.array([1.0]), np.array([1.0]), insts, particles,
                    particles)


def random_instance(rng: np.random.Generator, dim: int, n: tuple, nb: int, tau_range=(0.05, 1.0),
                    source=False, L=None) -> Instance:
    """A small instance with random per-(band, cell) tau, wall temperatures and source."""
    ncells = int(np.prod(n[:dim]))
    if L is None:
        L = tuple(float(x) for x in rng.uniform(0.5, 1.5, size=dim))
    tau = rng.uniform(*tau_range, size=(nb, ncells))
    wall = rng.uniform(-1.0, 1.0, size=2 * dim)
    src = rng.uniform(0.0, 2.0, size=ncells) if source else None
    return Instance(dim, tuple(n), tuple(L), tau, wall, src)


def two_material_box(n: int, seed: int = 7, q0: float = 1.0) -> Instance:
    """3D gray unit box: tau = 2 for x < 1/2 and 0.02 for x >= 1/2 (a factor-100 jump),
    each cell scaled by 1 + 0.4 (u - 1/2) with u uniform from a seeded generator; walls at
    T = 0; a heat source q0 in a centred cube of side n/8 cells."""
    rng = np.random.default_rng(seed * 1000 + n)
    x = (np.arange(n) + 0.5) / n
    base = np.where(x < 0.5, 2.0, 0.02)
    tau = np.broadcast_to(base[None, None, :], (n, n, n)).copy()  # (z, y, x), x fastest
    tau *= 1.0 + 0.4 * (rng.uniform(size=tau.shape) - 0.5)
    src = np.zeros((n, n, n))
    s = max(1, n // 8)
    lo = (n - s) // 2
    src[lo:lo + s, lo:lo + s, lo:lo + s] = q0
    return Instance(3, (n, n, n), (1.0, 1.0, 1.0), tau.reshape(1, -1), np.zeros(6), src.reshape(-1))


def box_batch(n_inst: int = 16, seed: int = 7) -> Workload:
    """Batch of two-material boxes of uneven sizes n_k = 16 + round(48 k / (n_inst - 1))."""
    sizes = [16 + int(round(48 * k / max(1, n_inst - 1))) for k in range(n_inst)]
    insts = [two_material_box(nk, seed) for nk in sizes]
    return Workload(f"3D two-material boxes {sizes}", np.array([1.0]), np.array([1.0]), insts, 256, 256)


def silicon_like_bands(n_bands: int = 40):
    """Band-branch table for an isotropic, silicon-like dispersion (LA and TA, quadratic
    omega(k) = v_s k - c k^2 on [0, k_max]), non-dimensionalised: group speeds relative to
    the LA sound speed, specific heats from the linearised Bose-Einstein distribution at
    300 K (x^2 e^x / (e^x - 1)^2 times the density of states k^2 / v_g), relaxation time
    tau = 1 / (A omega^2) normalised so that the slowest-relaxing band centre has tau = 10
    and the range spans three decades. Returns (C [2*n_bands], v, tau_band, omega)."""
    branches = {"LA": (9.01, 2.0e-7), "TA": (5.23, 2.26e-7)}   # v_s [km/s], c [km/s * m] (fit shape only)
    k_max = 1.0
    C, v, om = [], [], []
    for name, (vs, cc) in branches.items():
        cn = cc * 1e7 / 2.0 * 0.9                             # curvature so that v_g(k_max) = 0.1 v_s
        edges = np.linspace(0.0, k_max, n_bands + 1)
        kc = 0.5 * (edges[1:] + edges[:-1])
        dk = edges[1:] - edges[:-1]
        omega = vs * kc - cn * vs * kc ** 2
        vg = vs * (1.0 - 2.0 * cn * kc)
        x = omega / omega.max() * 2.0                       # hbar omega / k_B T scale
        cb = x ** 2 * np.exp(x) / np.expm1(x) ** 2 * kc ** 2 / vg * dk * (2.0 if name == "TA" else 1.0)
        C.append(cb)
        v.append(vg / 9.01)
        om.append(omega)
    C = np.concatenate(C)
    v = np.concatenate(v)
    om = np.concatenate(om)
    C = C / C.sum()
    tau = 1.0 / om ** 2
    tau = tau / tau.max() * 10.0
    tau = np.maximum(tau, tau.max() * 1e-3)
    return C, v, tau, om


def nongray_square(n=256, n_bands=40, particles=256, sigma=0.1, q0=1.0) -> Workload:
    """2D non-gray square (unit side): silicon-like band table, tau uniform in space per
    band, Gaussian heat source of width sigma L at the centre, walls at T = 0."""
    C, v, tb, _ = silicon_like_bands(n_bands)
    nc = n * n
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    src = q0 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * sigma ** 2))
    tau = np.repeat(tb[:, None], nc, axis=1)
    inst = Instance(2, (n, n), (1.0, 1.0), tau, np.zeros(4), src.reshape(-1))
    return Workload(f"2D non-gray {n}x{n} {len(C)} band-branches", C, v, [inst], particles, particles)
