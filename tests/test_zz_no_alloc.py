"""GPU test of the allocation-free correction solve (iugkp_diffusion_solve_noalloc).

That entry point is for callers that cannot allocate device memory (their GPU memory is
owned by another allocator, or an allocation's synchronisation is unaffordable): it keeps
its scratch in a static device array instead. Here it is called through the C ABI twice
in a row, on two different grids, and each answer is compared with the correction that
the regular entry point iugkp_newton_step computes for the same problem (both solve the
same finite-volume equation; cells are optically thin, so iugkp_newton_step applies the
correction undamped). This file is named so that pytest collects it last.
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
    nc = n[0] * n[1]
    taus = rng.uniform(0.5 * tau, tau, size=(1, nc))
    inst = WL.Instance(2, n, L, taus, rng.uniform(-1, 1, 4))
    s = Solver(GridSpec(2, n, L), inst.tau, [1.0], [1.0], inst.wall_T, None, particles_per_cell=64,
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
    hx, hy = inst.L[0] / inst.n[0], inst.L[1] / inst.n[1]
    V = hx * hy
    m = 1.0 / inst.tau[0]
    rhs = (g["R"].cpu().numpy() - T_n.cpu().numpy() * V * m) / V
    kappa = inst.tau[0] / 3.0
    return dT, rhs, kappa


def test_noalloc_solve_matches_newton_step_two_calls():
    from paper_2506_09465_gb300 import _lib as L
    lib = L.load()
    results = []
    for n, L_, tau, seed in (((32, 24), (1.0, 0.75), 0.2, 3), ((20, 40), (0.5, 1.0), 0.1, 4)):
        s, inst = _problem(n, L_, tau, seed)
        dT, rhs, kappa = _reference(s, inst)
        grid = L.Grid(2, n[0], n[1], 1, L_[0], L_[1], 1.0)
        k_dev = torch.as_tensor(kappa, device="cuda", dtype=torch.float64)
        r_dev = torch.as_tensor(rhs, device="cuda", dtype=torch.float64)
        x_dev = torch.full_like(r_dev, 7.0)  # garbage in the output: the solve must start from zero
        iters = ctypes.c_int(0)
        st = lib.iugkp_diffusion_solve_noalloc(ctypes.byref(grid), k_dev.data_ptr(), 1.0, r_dev.data_ptr(),
                                               x_dev.data_ptr(), 1e-13, 20000, ctypes.byref(iters),
                                               torch.cuda.current_stream().cuda_stream)
        L.check(st, None)
        x = x_dev.cpu().numpy()
        err = np.abs(x - dT).max() / np.abs(dT).max()
        assert iters.value > 0 and err < 1e-9, (n, iters.value, err)
        results.append(err)
    assert len(results) == 2


def test_noalloc_rejects_oversized_grid():
    from paper_2506_09465_gb300 import _lib as L
    lib = L.load()
    grid = L.Grid(2, 512, 512, 1, 1.0, 1.0, 1.0)
    one = torch.ones(4, device="cuda", dtype=torch.float64)
    st = lib.iugkp_diffusion_solve_noalloc(ctypes.byref(grid), one.data_ptr(), 1.0, one.data_ptr(), one.data_ptr(),
                                           1e-10, 10, None, None)
    assert st == 1
    assert b"IUGKP_NOALLOC_MAX_CELLS" in lib.iugkp_last_error(None)
