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
    wall_face_T: Optional[np.ndarray] = None  # [boundary faces] or None (walls uniform)

    def wall_faces(self):
        """Boundary faces per wall, in the order -x, +x, -y, +y, -z, +z (the faces of the wall
        normal to axis a run over the axes (a+1)%3, (a+2)%3, the first fastest)."""
        n = list(self.n) + [1] * (3 - len(self.n))
        return [n[(a + 1) % 3] * n[(a + 2) % 3] for a in range(self.dim) for _ in (0, 1)]

    def face_temperatures(self) -> np.ndarray:
        if self.wall_face_T is not None:
            return np.asarray(self.wall_face_T, dtype=np.float64)
        return np.concatenate([np.full(m, t) for m, t in zip(self.wall_faces(), self.wall_T)])

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


def jump_slab(case: str = "A", n: int = 100, particles: int = 8000) -> Workload:
    """1D gray film with a tau jump at x = L/2 (Sec. 4.2 shape): L = 1, C = |v| = 1,
    tau = 10 for x < L/2 and 0.1 (case A) or 1 (case B) for x > L/2, black walls at
    T = +1 (x = 0) and -1 (x = L)."""
    right = {"A": 0.1, "B": 1.0}[case]
    x = (np.arange(n) + 0.5) / n
    tau = np.where(x < 0.5, 10.0, right).reshape(1, n)
    inst = Instance(1, (n,), (1.0,), tau, np.array([1.0, -1.0]))
    return Workload(f"1D gray slab {n} cells tau 10 | {right}", np.array([1.0]), np.array([1.0]), [inst], particles,
                    particles)


def multiscale_slab(n: int = 100, particles: int = 8000, A1: float = 2.0, A2: float = 1.0) -> Workload:
    """1D gray film with a continuously varying relaxation time (Sec. 4.3 shape),
    tau(x) = 10^(|A1 sin(2 pi x / L)| - A2) at the cell centres; A1 = 2, A2 = 1 spans
    [0.1, 10]. L = 1, C = |v| = 1, black walls at T = +1 and -1."""
    x = (np.arange(n) + 0.5) / n
    tau = (10.0 ** (np.abs(A1 * np.sin(2.0 * np.pi * x)) - A2)).reshape(1, n)
    inst = Instance(1, (n,), (1.0,), tau, np.array([1.0, -1.0]))
    return Workload(f"1D gray multiscale slab {n} cells", np.array([1.0]), np.array([1.0]), [inst], particles,
                    particles)


def cavity(n=128, Kn=1.0, particles=1024) -> Workload:
    """2D gray square cavity (Sec. 4.4 shape): unit square, top wall T = 1, others 0."""
    inst = Instance(2, (n, n), (1.0, 1.0), np.full((1, n * n), Kn), np.array([0.0, 0.0, 0.0, 1.0]))
    return Workload(f"2D gray cavity {n}x{n} Kn={Kn}", np.array([1.0]), np.array([1.0]), [inst], particles, particles)


def hot_segment_rectangle(Kn: float = 10.0, nx: int = 100, ny: int = 50, particles: int = 200) -> Workload:
    """2D gray rectangle with a heated segment (Sec. 4.5 shape): L_x = 2 L_y = 5 L_1 with
    L_1 = 1, a segment of length L_1 centred on the top wall at T = 1, every other boundary
    face at T = 0, C = |v| = 1, tau = Kn (mean free path Kn L_1)."""
    Lx, Ly = 5.0, 2.5
    inst = Instance(2, (nx, ny), (Lx, Ly), np.full((1, nx * ny), Kn), np.zeros(4))
    ft = np.zeros(2 * ny + 2 * nx)
    xc = (np.arange(nx) + 0.5) * Lx / nx
    ft[2 * ny + nx:] = np.where(np.abs(xc - Lx / 2) < 0.5, 1.0, 0.0)   # top wall faces
    inst.wall_face_T = ft
    return Workload(f"2D gray rectangle {nx}x{ny} hot top segment Kn={Kn}", np.array([1.0]), np.array([1.0]), [inst],
                    particles, particles)


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


def silicon_like_bands(n_bands: int = 40, r: float = 0.1, tau_max: float = 10.0, decades: float = 3.0):
    """Band-branch table for an isotropic, silicon-like dispersion, non-dimensionalised.

    Two branches, LA (sound speed 1) and TA (5.23 / 9.01 of it, degeneracy 2), each with the
    quadratic fit omega(k) = v_s (k - (1 - r) k^2 / 2) on k in [0, 1], so that the group speed
    v_s (1 - (1 - r) k) falls to r v_s at the zone edge. Each branch is cut into n_bands equal
    k-intervals; a band's specific heat is the linearised Bose-Einstein weight
    x^2 e^x / (e^x - 1)^2 (x = omega / omega_T, omega_T = 0.5) times the density of states
    k^2 dk times the degeneracy, normalised to sum 1. Relaxation times tau = 1 / (A omega^2)
    with A set so that the longest is tau_max, clipped to span `decades` decades.
    Returns (C, v, tau, omega), each of length 2 n_bands (LA bands first)."""
    edges = np.linspace(0.0, 1.0, n_bands + 1)
    kc = 0.5 * (edges[1:] + edges[:-1])
    dk = np.diff(edges)
    C, v, om = [], [], []
    for vs, deg in ((1.0, 1.0), (5.23 / 9.01, 2.0)):
        omega = vs * (kc - 0.5 * (1.0 - r) * kc ** 2)
        vg = vs * (1.0 - (1.0 - r) * kc)
        x = omega / 0.5
        C.append(deg * x ** 2 * np.exp(x) / np.expm1(x) ** 2 * kc ** 2 * dk)
        v.append(vg)
        om.append(omega)
    C = np.concatenate(C)
    C = C / C.sum()
    v = np.concatenate(v)
    om = np.concatenate(om)
    tau = tau_max * (om.min() / om) ** 2
    tau = np.maximum(tau, tau_max * 10.0 ** (-decades))
    return C, v, tau, om


def nongray_square(n=256, n_bands=40, particles=1024, sigma=0.1, q0=1.0) -> Workload:
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


def nongray_batch(n_inst: int = 32, n_min: int = 64, n_max: int = 512, n_bands: int = 20, particles: int = 128,
                  sigma: float = 0.1, q0: float = 1.0) -> Workload:
    """Batch of non-gray squares of uneven sizes n_k = n_min (n_max / n_min)^(k / (n_inst - 1))
    rounded to even numbers, each with the silicon-like table of n_bands per branch, a
    Gaussian source of width sigma L at the centre and walls at T = 0."""
    C, v, tb, _ = silicon_like_bands(n_bands)
    insts = []
    for k in range(n_inst):
        nk = n_min * (n_max / n_min) ** (k / max(1, n_inst - 1))
        nk = int(2 * round(nk / 2))
        x = (np.arange(nk) + 0.5) / nk
        X, Y = np.meshgrid(x, x, indexing="xy")
        src = q0 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * sigma ** 2))
        insts.append(Instance(2, (nk, nk), (1.0, 1.0), np.repeat(tb[:, None], nk * nk, axis=1), np.zeros(4),
                              src.reshape(-1)))
    return Workload(f"2D non-gray batch of {n_inst} squares {insts[0].n[0]}..{insts[-1].n[0]}", C, v, insts,
                    particles, particles)


def hotspot_objective(inst: Instance, frac: float = 0.1) -> np.ndarray:
    """g with J = g . T the mean temperature over a centred square of `frac` of the area."""
    n = inst.n[0]
    side = max(1, int(round(n * np.sqrt(frac))))
    lo = (n - side) // 2
    g = np.zeros((inst.n[1], n))
    g[lo:lo + side, lo:lo + side] = 1.0
    return (g / g.sum()).reshape(-1)
