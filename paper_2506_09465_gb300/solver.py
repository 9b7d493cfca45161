"""Python front end of the IUGKP CUDA library: a context over one or several instances
(structured grids with their relaxation times, wall temperatures and sources), and thin
wrappers over each C-ABI call. Device memory and streams come from PyTorch; all the work
runs in libiugkp.so (arXiv 2506.09465: sweep Sec. 3.1-3.2, Newton step Sec. 3.3)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L


@dataclass
class GridSpec:
    """Uniform structured grid: dim in {1, 2, 3}, n cells per axis, L lengths."""
    dim: int
    n: Sequence[int]
    L: Sequence[float]

    def c(self) -> L.Grid:
        n = list(self.n) + [1] * (3 - len(self.n))
        ll = list(self.L) + [1.0] * (3 - len(self.L))
        return L.Grid(self.dim, n[0], n[1], n[2], ll[0], ll[1], ll[2])

    @property
    def ncells(self) -> int:
        return int(np.prod(list(self.n)[: self.dim]))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


class Solver:
    """A context holding one or more instances with a shared band table.

    grids: GridSpec or list of them (same dim); tau: array [nb, ncells] or list per instance;
    C, v: per band-branch; wall_T: [2*dim] or list; source: [ncells] power density, None, or
    list. options: keyword overrides of iugkp_options (see include/iugkp.h)."""

    def __init__(self, grids, tau, C, v, wall_T, source=None, device=None, **options):
        self.lib = L.load()
        if device is not None:
            torch.cuda.set_device(device)
        if isinstance(grids, GridSpec):
            grids, tau, wall_T, source = [grids], [tau], [wall_T], [source]
        n = len(grids)
        self.grids = list(grids)
        C = np.ascontiguousarray(C, dtype=np.float64).reshape(-1)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        self.nb = len(C)
        self._keep = []
        taus = [np.ascontiguousarray(t, dtype=np.float64).reshape(self.nb, -1) for t in tau]
        walls = [np.ascontiguousarray(w, dtype=np.float64).reshape(-1) for w in wall_T]
        if source is None:
            source = [None] * n
        srcs = [None if s is None else np.ascontiguousarray(s, dtype=np.float64).reshape(-1) for s in source]
        self._keep += [C, v, taus, walls, srcs]
        garr = (L.Grid * n)(*[g.c() for g in grids])
        tau_p = (ctypes.c_void_p * n)(*[t.ctypes.data for t in taus])
        wall_p = (ctypes.c_void_p * n)(*[w.ctypes.data for w in walls])
        src_p = (ctypes.c_void_p * n)(*[None if s is None else s.ctypes.data for s in srcs])
        bands = L.Bands(self.nb, C.ctypes.data, v.ctypes.data)
        self.options = L.default_options(**options)
        ctx = ctypes.c_void_p()
        st = self.lib.iugkp_create_batch(n, garr, ctypes.cast(tau_p, ctypes.c_void_p), ctypes.byref(bands),
                                         ctypes.cast(wall_p, ctypes.c_void_p), ctypes.cast(src_p, ctypes.c_void_p),
                                         ctypes.byref(self.options), ctypes.byref(ctx))
        L.check(st, None)
        self.ctx = ctx
        lay = L.Layout()
        co = (ctypes.c_longlong * (n + 1))()
        fo = (ctypes.c_longlong * (n + 1))()
        L.check(self.lib.iugkp_get_layout(self.ctx, ctypes.byref(lay), co, fo), self.ctx)
        self.layout = lay
        self.cell_off = list(co)
        self.face_off = list(fo)
        self.dim = lay.dim
        self.device = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.iugkp_destroy(ctx)
            self.ctx = None

    # -- sizes -----------------------------------------------------------------
    @property
    def total_cells(self) -> int:
        return self.layout.total_cells

    @property
    def total_faces(self) -> int:
        return self.layout.total_faces

    @property
    def total_walls(self) -> int:
        return self.layout.total_walls

    def zeros(self, n, dtype=torch.float64):
        return torch.zeros(n, dtype=dtype, device=self.device)

    # -- calls -------------------------------------------------------------------
    def sweep(self, T: torch.Tensor, epoch: int = 0, want_W=True, want_F=True, want_wall=True, stream=None):
        """One sweep from the cell temperatures T (device FP64). Returns dict of R, W, F, wall,
        counters (flights, candidates, real, crossings, wall exits, dropped)."""
        R = self.zeros(self.nb * self.total_cells)
        W = self.zeros(self.nb * self.total_cells) if want_W else None
        F = self.zeros(self.total_faces) if want_F else None
        wall = self.zeros(self.total_walls) if want_wall else None
        cnt = torch.zeros(6, dtype=torch.int64, device=self.device)
        st = self.lib.iugkp_sweep(self.ctx, _dptr(T), epoch, _dptr(R), _dptr(W), _dptr(F), _dptr(wall), _dptr(cnt),
                                  _stream_ptr(stream))
        L.check(st, self.ctx)
        return {"R": R, "W": W, "F": F, "wall": wall, "counters": cnt}

    def sweep_into(self, T, epoch, R, W=None, F=None, wall=None, counters=None, stream=None):
        st = self.lib.iugkp_sweep(self.ctx, _dptr(T), epoch, _dptr(R), _dptr(W), _dptr(F), _dptr(wall),
                                  _dptr(counters), _stream_ptr(stream))
        L.check(st, self.ctx)

    def macro(self, R, W=None, stream=None):
        T_half = self.zeros(self.total_cells)
        T_E = self.zeros(self.total_cells) if W is not None else None
        L.check(self.lib.iugkp_macro(self.ctx, _dptr(R), _dptr(W), _dptr(T_half), _dptr(T_E), _stream_ptr(stream)),
                self.ctx)
        return T_half, T_E

    def newton_step(self, T_n, T_half, R, stream=None) -> int:
        it = ctypes.c_int(0)
        L.check(self.lib.iugkp_newton_step(self.ctx, _dptr(T_n), _dptr(T_half), _dptr(R), _stream_ptr(stream),
                                           ctypes.byref(it)), self.ctx)
        return it.value

    def solve_steady(self, T0=None, tol=1e-8, max_iter=1000, stream=None, raise_on_noconv=True):
        T = self.zeros(self.total_cells) if T0 is None else T0.clone()
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        st = self.lib.iugkp_solve_steady(self.ctx, _dptr(T), tol, max_iter, ctypes.byref(it), ctypes.byref(res),
                                         _stream_ptr(stream))
        if st != 0 and (raise_on_noconv or st != 4):
            L.check(st, self.ctx)
        return T, it.value, res.value

    def adjoint(self, g, tol=1e-10, max_iter=500, stream=None):
        gs = self.zeros(self.total_cells)
        gw = self.zeros(self.total_walls)
        lam = self.zeros(self.total_cells)
        L.check(self.lib.iugkp_adjoint(self.ctx, None, _dptr(g), tol, max_iter, _dptr(gs), _dptr(gw), _dptr(lam),
                                       _stream_ptr(stream)), self.ctx)
        return gs, gw, lam

    def average(self, T, n_steps, epoch_first, want_var=True, want_F=False, stream=None):
        """Statistical averaging after convergence (iugkp_average): n_steps fresh-draw
        iterations from T (updated in place to the last iterate); returns (mean, var, F_mean)."""
        mean = self.zeros(self.total_cells)
        var = self.zeros(self.total_cells) if want_var else None
        Fm = self.zeros(self.total_faces) if want_F else None
        L.check(self.lib.iugkp_average(self.ctx, _dptr(T), int(n_steps), int(epoch_first), _dptr(mean), _dptr(var),
                                       _dptr(Fm), _stream_ptr(stream)), self.ctx)
        return mean, var, Fm

    def persistent_reset(self, stream=None):
        """(Re)builds the persistent null-collision population (iugkp_persistent_reset)."""
        L.check(self.lib.iugkp_persistent_reset(self.ctx, _stream_ptr(stream)), self.ctx)

    def persistent_step(self, T, iteration, stream=None):
        """One iteration of the persistent population (iugkp_persistent_step): returns
        dict(R, W, wall, counters, slots)."""
        R = self.zeros(self.nb * self.total_cells)
        W = self.zeros(self.nb * self.total_cells)
        wall = self.zeros(self.total_walls)
        cnt = torch.zeros(6, dtype=torch.int64, device=self.device)
        n = ctypes.c_longlong(0)
        L.check(self.lib.iugkp_persistent_step(self.ctx, _dptr(T), int(iteration), _dptr(R), _dptr(W), _dptr(wall),
                                               _dptr(cnt), ctypes.byref(n), _stream_ptr(stream)), self.ctx)
        return {"R": R, "W": W, "wall": wall, "counters": cnt, "slots": n.value}

    def autotune(self, T, epoch=0, allow_k32=False, stream=None):
        """Times the staged sweep over its tunables and keeps the fastest (see iugkp_autotune)."""
        t = L.Tuning()
        L.check(self.lib.iugkp_autotune(self.ctx, _dptr(T), epoch, int(allow_k32), ctypes.byref(t),
                                        _stream_ptr(stream)), self.ctx)
        return {"refill_lanes": t.refill_lanes, "warp_grab": t.warp_grab, "walk_k": t.walk_k, "tally": t.tally,
                "sweep_ms": t.sweep_ms, "baseline_ms": t.baseline_ms}

    def replayed(self, stream=None) -> int:
        """Particles of the last staged sweep (or adjoint re-trace) the FP64 walk replayed."""
        n = ctypes.c_longlong(0)
        L.check(self.lib.iugkp_replayed(self.ctx, ctypes.byref(n), _stream_ptr(stream)), self.ctx)
        return n.value

    def set_source(self, Q, stream=None):
        self._set(L.FIELD_SOURCE, Q, stream)

    def set_wall_T(self, Tw, stream=None):
        self._set(L.FIELD_WALL_T, Tw, stream)

    def set_tau(self, tau, stream=None):
        """Relaxation times [instance][band][cell] (rebuilds every tau-dependent part)."""
        self._set(L.FIELD_TAU, tau, stream)
        L.check(self.lib.iugkp_get_layout(self.ctx, ctypes.byref(self.layout), None, None), self.ctx)

    def set_wall_face_T(self, Tf, stream=None):
        """Temperature of every boundary face ([total_wall_faces], instance-major)."""
        self._set(L.FIELD_WALL_FACE_T, Tf, stream)

    def _set(self, which, data, stream):
        if isinstance(data, torch.Tensor) and data.is_cuda:
            d = data.to(torch.float64).contiguous()
            st = self.lib.iugkp_set_field(self.ctx, which, d.data_ptr(), 1, _stream_ptr(stream))
        else:
            a = np.ascontiguousarray(np.asarray(data, dtype=np.float64).reshape(-1))
            st = self.lib.iugkp_set_field(self.ctx, which, a.ctypes.data, 0, _stream_ptr(stream))
        L.check(st, self.ctx)


class IugkpSteady(torch.autograd.Function):
    """T* = steady state as a function of (per-cell source Q, wall temperatures), with the
    frozen-draw adjoint (re-traced sweeps) as its backward."""

    @staticmethod
    def forward(ctx, source: torch.Tensor, wall_T: torch.Tensor, solver: Solver, tol: float = 1e-10,
                max_iter: int = 1000):
        solver.set_source(source.detach())
        solver.set_wall_T(wall_T.detach())
        T, _, _ = solver.solve_steady(None, tol, max_iter)
        ctx.solver = solver
        ctx.tol = tol
        ctx.max_iter = max_iter
        return T

    @staticmethod
    def backward(ctx, grad_T):
        gs, gw, _ = ctx.solver.adjoint(grad_T.contiguous().to(torch.float64), ctx.tol, ctx.max_iter)
        return gs, gw, None, None, None
