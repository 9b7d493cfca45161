"""GPU test of the allocation-free correction solve (iugkp_diffusion_solve_noalloc).

That entry point is for callers that cannot allocate device memory (their GPU memory is
owned by another allocator, or an allocation's synchronisation is unaffordable): it keeps
its scratch in a static device array instead. Here it is called through the C ABI twice
in a row on two different 2D grids, then on a 1D and a 3D grid, and each answer is
compared with the correction that the regular entry point iugkp_newton_step computes for
the same problem (both solve the same finite-volume equation; cells are optically thin, so
iugkp_newton_step applies the correction undamped). Bad input (a kappa that is not
positive) is rejected with IUGKP_EINVAL. This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, L, tau, seed):
    from paper_2506_09465_gb300 import workloads as WL
    from paper_2506_09465_gb300.solver import GridSpec, Solver
    rng = np.random.default_rng(seed)
    dim = len(n)
    nc = int(np.prod(n))
    taus = rng.uniform(0.5 * tau, tau, size=(1, nc))
    inst = WL.Instance(dim, n, L, taus, rng.uniform(-1, 1, 2 * dim))
    s = Solver(GridSpec(dim, n, L), inst.tau, [1.0], [1.0], inst.wall_T, None, particles_per_cell=64,
               particles_per_wall_face=64, cg_rtol=1e-13, cg_maxit=20000)
    return s, inst


def _reference(s, inst):
    """Correction computed by iugkp_newton_step, and the Newton source it solved for."""
    T_n = torch.as_tensor(np.random.default_rng(1).uniform(0, 1, inst.ncells), device="cuda")
    g = s.sweep(T_n, 0)
    T_half, _ = s.macro(g["R"])
    before = T_half.clone()
    s.newton_step(T_n, T_half, g["R"])
    dT = (T_half - before).cpu().numpy()
    V = float(np.prod([inst.L[a] / inst.n[a] for a in range(inst.dim)]))
    m = 1.0 / inst.tau[0]
    rhs = (g["R"].cpu().numpy() - T_n.cpu().numpy() * V * m) / V
    kappa = inst.tau[0] / 3.0
    return dT, rhs, kappa


def _grid(L, n, Ls):
    nn = list(n) + [1] * (3 - len(n))
    ll = list(Ls) + [1.0] * (3 - len(Ls))
    return L.Grid(len(n), nn[0], nn[1], nn[2], ll[0], ll[1], ll[2])


def _solve(lib, L, n, Ls, kappa, rhs):
    grid = _grid(L, n, Ls)
    k_dev = torch.as_tensor(kappa, device="cuda", dtype=torch.float64)
    r_dev = torch.as_tensor(rhs, device="cuda", dtype=torch.float64)
    x_dev = torch.full_like(r_dev, 7.0)  # garbage in the output: the solve must start from zero
    iters = ctypes.c_int(0)
    st = lib.iugkp_diffusion_solve_noalloc(ctypes.byref(grid), k_dev.data_ptr(), 1.0, r_dev.data_ptr(),
                                           x_dev.data_ptr(), 1e-13, 20000, ctypes.byref(iters),
                                           torch.cuda.current_stream().cuda_stream)
    return st, iters.value, x_dev.cpu().numpy()


@pytest.mark.parametrize("cases", [
    (((32, 24), (1.0, 0.75), 0.2, 3), ((20, 40), (0.5, 1.0), 0.1, 4)),   # two calls in a row, 2D
    (((30,), (1.0,), 0.2, 5), ((6, 5, 4), (1.0, 1.0, 1.0), 1.0, 6)),     # 1D, then 3D
])
def test_noalloc_solve_matches_newton_step(cases):
    from paper_2506_09465_gb300 import _lib as L
    lib = L.load()
    for n, Ls, tau, seed in cases:
        s, inst = _problem(n, Ls, tau, seed)
        dT, rhs, kappa = _reference(s, inst)
        st, it, x = _solve(lib, L, n, Ls, kappa, rhs)
        L.check(st, None)
        err = np.abs(x - dT).max() / np.abs(dT).max()
        assert it > 0 and err < 1e-9, (n, it, err)


def test_noalloc_rejects_bad_input():
    from paper_2506_09465_gb300 import _lib as L
    lib = L.load()
    grid = L.Grid(2, 512, 512, 1, 1.0, 1.0, 1.0)
    one = torch.ones(4, device="cuda", dtype=torch.float64)
    st = lib.iugkp_diffusion_solve_noalloc(ctypes.byref(grid), one.data_ptr(), 1.0, one.data_ptr(), one.data_ptr(),
                                           1e-10, 10, None, None)
    assert st == 1
    assert b"IUGKP_NOALLOC_MAX_CELLS" in lib.iugkp_last_error(None)
    # a zero conductivity: rejected after the stencil pass, before any iteration
    kappa = np.full(12 * 10, 0.1)
    kappa[17] = 0.0
    st, it, _ = _solve(lib, L, (12, 10), (1.0, 1.0), kappa, np.ones(120))
    assert st == 1 and it == -2
    assert b"kappa" in lib.iugkp_last_error(None)
    # and a good call right after still works
    st, it, x = _solve(lib, L, (12, 10), (1.0, 1.0), np.full(120, 0.1), np.ones(120))
    assert st == 0 and it > 0 and np.all(np.isfinite(x))
