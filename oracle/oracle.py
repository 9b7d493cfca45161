"""Python access to the FP64 CPU oracle (``iugkp_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference legs may import this module. It shares no
code with the CUDA path and does not import the product package.

Every function restates a step of the IUGKP method of Liu, Yang, Zhang, Ji and Xu
(arXiv 2506.09465); the C++ file names the section or equation it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iugkp_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain g++, FP64, no
    fused multiply-add)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("nb", ctypes.c_int),
        ("C", ctypes.c_void_p), ("v", ctypes.c_void_p), ("tau", ctypes.c_void_p),
        ("wall_T", ctypes.c_void_p), ("source", ctypes.c_void_p),
        ("n_band", ctypes.c_void_p), ("n_wall_band", ctypes.c_void_p),
        ("seed", ctypes.c_ulonglong), ("instance", ctypes.c_uint), ("budget", ctypes.c_longlong),
        ("wall_face_T", ctypes.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        vp, d, u32, i32, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_uint32, ctypes.c_int, ctypes.c_longlong
        _lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
        _lib.orc_word_to_uniform.argtypes = [u32]
        _lib.orc_word_to_uniform.restype = d
        _lib.orc_stream.argtypes = [ctypes.c_ulonglong, u32, u32, u32, u32, u32, i64, vp]
        _lib.orc_ncells.argtypes = [P]
        _lib.orc_ncells.restype = i64
        _lib.orc_nfaces.argtypes = [P]
        _lib.orc_nfaces.restype = i64
        _lib.orc_sweep.argtypes = [P, vp, u32, vp, vp, vp, vp, vp]
        _lib.orc_macro.argtypes = [P, vp, vp, vp, vp]
        _lib.orc_diffusion_apply.argtypes = [P, vp, vp]
        _lib.orc_diffusion_solve.argtypes = [P, vp, vp]
        _lib.orc_newton.argtypes = [P, vp, vp, vp, vp]
        _lib.orc_residual.argtypes = [i64, vp, vp, d]
        _lib.orc_residual.restype = d
        _lib.orc_solve_steady.argtypes = [P, vp, d, i32, i32, u32, i32, d, vp, vp, vp]
        _lib.orc_adjoint_apply.argtypes = [P, vp, u32, vp, vp]
        _lib.orc_band_split.argtypes = [i32, i64, vp, vp]
        _lib.orc_emit.argtypes = [P, i32, i32, i64, u32, vp, vp, vp]
        _lib.orc_newton_theta.argtypes = [P]
        _lib.orc_newton_theta.restype = d
        _lib.orc_persistent_step.argtypes = [P, vp, u32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc_persistent_step.restype = i32
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


@dataclass
class Problem:
    """One IUGKP instance for the oracle (all host FP64 arrays).

    dim, n = (nx, ny, nz), L = (lx, ly, lz): uniform structured grid on [0, L];
    C, v: per band-branch; tau: [nb, ncells] (x fastest); wall_T: [2*dim] in the order
    -x, +x, -y, +y, -z, +z; source: [ncells] power density or None;
    n_band / n_wall_band: particles per cell / per boundary face for each band;
    wall_face_T: temperature of every boundary face (walls in wall_T order; on the wall
    normal to axis a the faces run over axes (a+1)%3, (a+2)%3, the first fastest), or None.
    """
    dim: int
    n: Sequence[int]
    L: Sequence[float]
    C: np.ndarray
    v: np.ndarray
    tau: np.ndarray
    wall_T: np.ndarray
    n_band: np.ndarray
    n_wall_band: np.ndarray
    source: Optional[np.ndarray] = None
    seed: int = 0
    instance: int = 0
    budget: int = 1 << 24
    wall_face_T: Optional[np.ndarray] = None
    _keep: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        n = list(self.n) + [1] * (3 - len(self.n))
        L = list(self.L) + [1.0] * (3 - len(self.L))
        self.n, self.L = tuple(int(x) for x in n), tuple(float(x) for x in L)
        self.C = np.ascontiguousarray(self.C, dtype=np.float64)
        self.v = np.ascontiguousarray(self.v, dtype=np.float64)
        self.tau = np.ascontiguousarray(self.tau, dtype=np.float64).reshape(len(self.C), -1)
        self.wall_T = np.ascontiguousarray(self.wall_T, dtype=np.float64)
        self.n_band = np.ascontiguousarray(self.n_band, dtype=np.int64)
        self.n_wall_band = np.ascontiguousarray(self.n_wall_band, dtype=np.int64)
        if self.source is not None:
            self.source = np.ascontiguousarray(self.source, dtype=np.float64)
        if self.wall_face_T is not None:
            self.wall_face_T = np.ascontiguousarray(self.wall_face_T, dtype=np.float64)

    @property
    def nb(self) -> int:
        return len(self.C)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def c_struct(self) -> _Problem:
        s = _Problem()
        s.dim = self.dim
        s.nx, s.ny, s.nz = self.n
        s.lx, s.ly, s.lz = self.L
        s.nb = self.nb
        s.C, s.v, s.tau = _ptr(self.C), _ptr(self.v), _ptr(self.tau)
        s.wall_T, s.source = _ptr(self.wall_T), _ptr(self.source)
        s.n_band, s.n_wall_band = _ptr(self.n_band), _ptr(self.n_wall_band)
        s.seed, s.instance, s.budget = self.seed, self.instance, self.budget
        s.wall_face_T = _ptr(self.wall_face_T)
        return s

    def wall_faces(self):
        """Boundary faces per wall, in wall order."""
        n = self.n
        return [n[(a + 1) % 3] * n[(a + 2) % 3] for a in range(self.dim) for _ in (0, 1)]

    def nfaces(self) -> int:
        return int(lib().orc_nfaces(ctypes.byref(self.c_struct())))

    def face_counts(self):
        """Faces normal to each axis (x-faces first, then y, then z)."""
        n = self.n
        out = []
        for a in range(3):
            if a < self.dim:
                m = [n[0], n[1], n[2]]
                m[a] += 1
                out.append(m[0] * m[1] * m[2])
            else:
                out.append(0)
        return out

    def h(self):
        return tuple(self.L[a] / self.n[a] if a < self.dim else 1.0 for a in range(3))

    def volume(self) -> float:
        hx, hy, hz = self.h()
        return hx * hy * hz


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def word_to_uniform(a: int) -> float:
    return float(lib().orc_word_to_uniform(int(a)))


def stream(seed, instance, band, epoch, emitter, particle, n) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    lib().orc_stream(seed, instance, band, epoch, emitter, particle, n, _ptr(out))
    return out


@dataclass
class SweepResult:
    R: np.ndarray       # [nb, ncells] real-collision power (W^h)
    W: np.ndarray       # [nb, ncells] candidate estimator of energy (W)
    F: np.ndarray       # [nfaces] net power across each face, +axis direction
    wall: np.ndarray    # [2*dim] absorbed power per wall
    counters: np.ndarray  # flights, candidates, real, crossings, wall exits, dropped


def sweep(p: Problem, T: np.ndarray, epoch: int = 0) -> SweepResult:
    T = np.ascontiguousarray(T, dtype=np.float64)
    assert T.size == p.ncells
    R = np.zeros((p.nb, p.ncells))
    W = np.zeros((p.nb, p.ncells))
    F = np.zeros(p.nfaces())
    wall = np.zeros(2 * p.dim)
    cnt = np.zeros(6, dtype=np.uint64)
    rc = lib().orc_sweep(ctypes.byref(p.c_struct()), _ptr(T), epoch, _ptr(R), _ptr(W), _ptr(F), _ptr(wall), _ptr(cnt))
    if rc != 0:
        raise ValueError(f"orc_sweep failed ({rc})")
    return SweepResult(R, W, F, wall, cnt)


def macro(p: Problem, R: np.ndarray, W: np.ndarray):
    T_half = np.zeros(p.ncells)
    T_E = np.zeros(p.ncells)
    R = np.ascontiguousarray(R, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    rc = lib().orc_macro(ctypes.byref(p.c_struct()), _ptr(R), _ptr(W), _ptr(T_half), _ptr(T_E))
    if rc != 0:
        raise ValueError("orc_macro failed")
    return T_half, T_E


def diffusion_apply(p: Problem, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(p.ncells)
    lib().orc_diffusion_apply(ctypes.byref(p.c_struct()), _ptr(x), _ptr(y))
    return y


def diffusion_solve(p: Problem, rhs: np.ndarray) -> np.ndarray:
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.zeros(p.ncells)
    rc = lib().orc_diffusion_solve(ctypes.byref(p.c_struct()), _ptr(rhs), _ptr(x))
    if rc != 0:
        raise ValueError("diffusion solve failed")
    return x


def newton(p: Problem, T_n: np.ndarray, T_half: np.ndarray, R: np.ndarray):
    """Returns (T_{n+1}, dT)."""
    T_n = np.ascontiguousarray(T_n, dtype=np.float64)
    out = np.array(T_half, dtype=np.float64, copy=True)
    dT = np.zeros(p.ncells)
    R = np.ascontiguousarray(R, dtype=np.float64)
    rc = lib().orc_newton(ctypes.byref(p.c_struct()), _ptr(T_n), _ptr(out), _ptr(R), _ptr(dT))
    if rc != 0:
        raise ValueError("orc_newton failed")
    return out, dT


def newton_theta(p: Problem) -> float:
    """Damping of the correction, min(1, 1.5 / optical thickness of the thickest cell)."""
    return float(lib().orc_newton_theta(ctypes.byref(p.c_struct())))


def residual(T0: np.ndarray, T1: np.ndarray, dT_ref: float) -> float:
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    T1 = np.ascontiguousarray(T1, dtype=np.float64)
    return float(lib().orc_residual(T0.size, _ptr(T0), _ptr(T1), dT_ref))


def solve_steady(p: Problem, T0: np.ndarray, tol: float, max_iter: int, frozen: bool = True,
                 epoch0: int = 0, newton: bool = False, dT_ref: float = 1.0):
    """Returns (T, iterations, final residual, residual history)."""
    T = np.array(T0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    hist = np.zeros(max_iter)
    rc = lib().orc_solve_steady(ctypes.byref(p.c_struct()), _ptr(T), tol, max_iter, int(frozen), epoch0,
                                int(newton), dT_ref, ctypes.byref(it), ctypes.byref(res), _ptr(hist))
    if rc != 0:
        raise ValueError(f"orc_solve_steady failed ({rc})")
    return T, it.value, res.value, hist[: it.value]


def average(p: Problem, T0: np.ndarray, n_steps: int, epoch_first: int, newton_on: bool = True):
    """Statistical averaging after convergence (Sec. 4.4-4.5: extra steps whose results are
    averaged to reduce the statistical noise): n_steps further iterations, each with fresh
    draws (epoch = epoch_first + step) and the same update as the solve (sweep, macro
    update, Newton correction); returns the last iterate, the mean and the sample variance
    (n - 1 in the denominator) of the n_steps iterates, and the mean face power.
    Plain two-pass statistics over the stored iterates."""
    T = np.array(T0, dtype=np.float64, copy=True)
    Ts, Fs = [], []
    for k in range(n_steps):
        r = sweep(p, T, epoch_first + k)
        T_half, _ = macro(p, r.R, r.W)
        T = newton(p, T, T_half, r.R)[0] if newton_on else T_half
        Ts.append(T.copy())
        Fs.append(r.F.copy())
    Ts = np.array(Ts)
    var = Ts.var(axis=0, ddof=1) if n_steps > 1 else np.zeros(p.ncells)
    return T, Ts.mean(axis=0), var, np.array(Fs).mean(axis=0)


class Population:
    """Fixed particle population of the persistent null-collision scheme (Sec. 3.2 steps
    (1)-(6)): per slot position, direction, weight, band, home (cell, or ncells + boundary
    face in wall order) and whether it is re-emitted this iteration; with the number of
    particles that ended at each home in the last iteration."""

    def __init__(self, p: Problem):
        nc, nb = p.ncells, p.nb
        nbf = sum(p.wall_faces())
        slots_b, homes = [], []
        # slot q * ncells + cell of each band, then q * faces + face (q-major)
        for b in range(nb):
            slots_b.append(np.full(int(p.n_band[b]) * nc, b))
            homes.append(np.tile(np.arange(nc), int(p.n_band[b])))
        for b in range(nb):
            slots_b.append(np.full(int(p.n_wall_band[b]) * nbf, b))
            homes.append(nc + np.tile(np.arange(nbf), int(p.n_wall_band[b])))
        self.band = np.ascontiguousarray(np.concatenate(slots_b), dtype=np.int32)
        self.home = np.ascontiguousarray(np.concatenate(homes), dtype=np.int64)
        self.n = len(self.band)
        self.x = np.zeros(3 * self.n)
        self.s = np.zeros(3 * self.n)
        self.w = np.zeros(self.n)
        self.due = np.ones(self.n, dtype=np.int32)
        # step (1): every home starts with its own N particles
        counts = np.zeros((nb, nc + nbf), dtype=np.uint32)
        for b in range(nb):
            counts[b, :nc] = p.n_band[b]
            counts[b, nc:] = p.n_wall_band[b]
        self.n_home = counts.reshape(-1)


def persistent_step(p: Problem, T: np.ndarray, it: int, pop: Population):
    """One iteration of the persistent scheme: returns (R, W, wall, counters); pop is
    updated in place."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    R = np.zeros((p.nb, p.ncells))
    W = np.zeros((p.nb, p.ncells))
    wall = np.zeros(2 * p.dim)
    cnt = np.zeros(6, dtype=np.uint64)
    n_new = np.zeros_like(pop.n_home)
    rc = lib().orc_persistent_step(ctypes.byref(p.c_struct()), _ptr(T), it, pop.n, _ptr(pop.x), _ptr(pop.s),
                                   _ptr(pop.w), _ptr(pop.band), _ptr(pop.home), _ptr(pop.due), _ptr(pop.n_home),
                                   _ptr(n_new), _ptr(R), _ptr(W), _ptr(wall), _ptr(cnt))
    if rc != 0:
        raise ValueError("orc_persistent_step failed")
    pop.n_home = n_new
    return R, W, wall, cnt


def adjoint_apply(p: Problem, lam: np.ndarray, epoch: int = 0):
    """Returns (A^T lam over cells, B_wall^T lam per wall) for one sweep's draws."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.zeros(p.ncells)
    gw = np.zeros(2 * p.dim)
    rc = lib().orc_adjoint_apply(ctypes.byref(p.c_struct()), _ptr(lam), epoch, _ptr(out), _ptr(gw))
    if rc != 0:
        raise ValueError("orc_adjoint_apply failed")
    return out, gw


def emit(p: Problem, kind: int, band: int, emitter: int, epoch: int = 0):
    """Start states (x [N,3], s [N,3], first path length d [N]) of one emitter's
    particles: kind 0 = cell `emitter`, kind 1 = boundary face `emitter`."""
    N = int(p.n_band[band] if kind == 0 else p.n_wall_band[band])
    x = np.zeros((N, 3))
    s = np.zeros((N, 3))
    d = np.zeros(N)
    k = lib().orc_emit(ctypes.byref(p.c_struct()), kind, band, emitter, epoch, _ptr(x), _ptr(s), _ptr(d))
    if k != N:
        raise ValueError(f"orc_emit returned {k}, expected {N}")
    return x, s, d


def band_split(N: int, r: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(len(r), dtype=np.int64)
    rc = lib().orc_band_split(len(r), N, _ptr(r), _ptr(out))
    if rc != 0:
        raise ValueError("band split needs N >= nb and r > 0")
    return out


# ---------------------------------------------------------------------------
# Dense linear-algebra views of the frozen-draw iteration (tiny grids only).
# With the draws fixed, one sweep followed by the macro update is an affine map
# T_half = A T + b (Sec. 2, Eq. "sum-g": a convex combination of equilibria).
# ---------------------------------------------------------------------------

def cell_m(p: Problem) -> np.ndarray:
    """m_i = sum_b C_b / tau_{b,i}."""
    return (p.C[:, None] / p.tau).sum(axis=0)


def assemble_affine(p: Problem, epoch: int = 0):
    """Columns of A (unit T in one cell, walls 0, no source) and of B_wall (unit
    temperature on one wall), each by one oracle sweep."""
    n = p.ncells
    q = Problem(p.dim, p.n, p.L, p.C, p.v, p.tau, np.zeros(2 * p.dim), p.n_band, p.n_wall_band,
                None, p.seed, p.instance, p.budget)
    A = np.zeros((n, n))
    for j in range(n):
        T = np.zeros(n)
        T[j] = 1.0
        r = sweep(q, T, epoch)
        A[:, j] = macro(q, r.R, r.W)[0]
    Bw = np.zeros((n, 2 * p.dim))
    for w in range(2 * p.dim):
        q.wall_T = np.zeros(2 * p.dim)
        q.wall_T[w] = 1.0
        r = sweep(q, np.zeros(n), epoch)
        Bw[:, w] = macro(q, r.R, r.W)[0]
    return A, Bw


def adjoint_dense(p: Problem, g: np.ndarray, epoch: int = 0):
    """Adjoint gradient of J = g . T* on a tiny grid by dense transposes.

    T* solves T = A (T + Q/m) + B_wall T_w (frozen draws; the source enters as an
    emission-temperature shift Q/m). lambda = (I - A^T)^{-1} g, then
    dJ/dQ = (A^T lambda) / m = (lambda - g) / m and dJ/dT_w = B_wall^T lambda.
    Returns (grad_source, grad_wall, lambda, A, B_wall).
    """
    A, Bw = assemble_affine(p, epoch)
    lam = np.linalg.solve(np.eye(p.ncells) - A.T, g)
    return (lam - g) / cell_m(p), Bw.T @ lam, lam, A, Bw


def adjoint_iterative(p: Problem, g: np.ndarray, epoch: int = 0, tol: float = 1e-12, max_iter: int = 500,
                      newton: bool = True):
    """Same gradient by re-tracing sweeps: lambda <- A^T lambda + g, with the transposed
    diffusion correction lambda += theta m D^{-1}(lambda_half - lambda) (the forward step
    is T += theta D^{-1} m (T_half - T); D is symmetric). Returns (grad_source, grad_wall,
    lambda, iters)."""
    m = cell_m(p)
    theta = newton_theta(p)
    lam = np.zeros(p.ncells)
    it = 0
    for it in range(1, max_iter + 1):
        at, _ = adjoint_apply(p, lam, epoch)
        half = at + g
        new = half + theta * m * diffusion_solve(p, half - lam) if newton else half
        res = residual(lam, new, float(np.abs(g).max()))
        lam = new
        if res <= tol:
            break
    at, gw = adjoint_apply(p, lam, epoch)
    return at / m, gw, lam, it
