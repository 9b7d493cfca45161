"""Shared helpers of the GPU tests: build the oracle problem and the CUDA solver from the
same seeded instance (each side computes its own band split and coefficients)."""
import numpy as np

from oracle import oracle as O


def oracle_problem(inst, C, v, N, Nw, seed=0, instance=0):
    C = np.asarray(C, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    r = C * (1.0 / inst.tau).mean(axis=1)
    n_band = O.band_split(N, r) if len(C) > 1 else np.array([N])
    n_wall = O.band_split(Nw, C * v) if len(C) > 1 else np.array([Nw])
    return O.Problem(inst.dim, inst.n, inst.L, C, v, inst.tau, inst.wall_T, n_band, n_wall,
                     source=inst.source, seed=seed, instance=instance,
                     wall_face_T=getattr(inst, "wall_face_T", None))


def gpu_solver(insts, C, v, N, Nw, **opt):
    from paper_2506_09465_gb300.solver import GridSpec, Solver
    if not isinstance(insts, (list, tuple)):
        insts = [insts]
    grids = [GridSpec(i.dim, i.n, i.L) for i in insts]
    s = Solver(grids, [i.tau for i in insts], C, v, [i.wall_T for i in insts], [i.source for i in insts],
               particles_per_cell=N, particles_per_wall_face=Nw, **opt)
    if any(getattr(i, "wall_face_T", None) is not None for i in insts):
        s.set_wall_face_T(np.concatenate([i.face_temperatures() for i in insts]))
    return s


def normwise_close(gpu, ora, rtol):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ora = np.asarray(ora, dtype=np.float64).ravel()
    scale = max(np.abs(ora).max(), 1e-300)
    err = np.abs(gpu - ora).max() / scale
    return err <= rtol, err
