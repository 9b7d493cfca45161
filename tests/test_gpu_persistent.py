"""The persistent null-collision population of Sec. 3.2 on the GPU (FP64): the same draws
and the same update as the oracle's, iteration after iteration; and with the paper's 8000
particles per cell its stationary energy temperature reproduces the expected steady state
of the stateless sweep across the tau jump of Case A and the multiscale film (Sec. 4.2-4.3)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_09465_gb300 import workloads as WL  # noqa: E402
from gpu_helpers import gpu_solver, normwise_close, oracle_problem  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def cuda(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def test_persistent_population_matches_oracle(orc):
    rng = np.random.default_rng(21)
    inst = WL.random_instance(rng, 2, (10, 7), 2, (0.05, 0.6), source=True)
    C, v = np.array([0.7, 1.3]), np.array([1.0, 0.6])
    p = oracle_problem(inst, C, v, 40, 24, seed=6)
    pop = orc.Population(p)
    s = gpu_solver(inst, C, v, 40, 24, precision=0, tally=0, schedule=0, seed=6)
    s.persistent_reset()
    T = rng.uniform(0.0, 1.0, inst.ncells)
    for it in range(5):
        R, W, wall, cnt = orc.persistent_step(p, T, it, pop)
        g = s.persistent_step(cuda(T), it)
        assert g["slots"] == pop.n
        for key, ref in (("R", R), ("W", W), ("wall", wall)):
            ok, err = normwise_close(g[key].cpu().numpy(), ref, 1e-10)
            assert ok, (it, key, err)
        assert g["counters"].cpu().numpy().tolist() == cnt.astype(np.int64).tolist(), it
        Th, _ = orc.macro(p, R, W)
        T = orc.newton(p, T, Th, R)[0]


def test_persistent_population_fp32_tracks_the_oracle(orc):
    # FP32 positions, directions and paths (FP64 weights and tallies): the same draws; a
    # particle changes cell only when it stops within FP32 rounding of a face, so the first
    # iterations agree with the oracle far below the statistical noise.
    rng = np.random.default_rng(22)
    inst = WL.random_instance(rng, 2, (12, 9), 1, (0.05, 0.6), source=True)
    p = oracle_problem(inst, [1.0], [1.0], 64, 64, seed=7)
    pop = orc.Population(p)
    s = gpu_solver(inst, [1.0], [1.0], 64, 64, seed=7)   # FP32 tracking (default)
    s.persistent_reset()
    T = rng.uniform(0.0, 1.0, inst.ncells)
    for it in range(2):
        R, W, wall, cnt = orc.persistent_step(p, T, it, pop)
        g = s.persistent_step(cuda(T), it)
        for key, ref in (("R", R), ("W", W), ("wall", wall)):
            ok, err = normwise_close(g[key].cpu().numpy(), ref, 2e-3)
            assert ok, (it, key, err)
        c_g = g["counters"].cpu().numpy().astype(float)
        assert np.all(np.abs(c_g - cnt.astype(float)) <= 1e-3 * cnt + 2), it
        T = orc.macro(p, R, W)[0]


@pytest.mark.parametrize("case,precision", [("caseA", 0), ("multiscale", 0), ("caseA", 1)])
def test_persistent_stationary_state_is_the_expected_steady_state(case, precision):
    name = {"caseA": "slab_jump_caseA_100cells.txt", "multiscale": "slab_multiscale_100cells.txt"}[case]
    wl = WL.jump_slab("A", 100, 8000) if case == "caseA" else WL.multiscale_slab(100, 8000)
    inst = wl.instances[0]
    Tg = np.array([float(l.split()[2]) for l in open(os.path.join(GOLDEN, name)) if l[0] != "#"])
    s = gpu_solver(inst, wl.C, wl.v, 8000, 8000, precision=precision, tally=0, schedule=0, seed=12)
    s.persistent_reset()
    T = torch.zeros(inst.ncells, dtype=torch.float64, device="cuda")
    hist = []
    for it in range(400):
        # the scheme's own update T = W^h / (V m)
        g = s.persistent_step(T, it)
        T, TE = s.macro(g["R"], g["W"])
        if it >= 200:
            hist.append(TE.cpu().numpy())
    bm = np.array(hist).reshape(20, 10, -1).mean(1)
    z = (bm.mean(0) - Tg) / (bm.std(0, ddof=1) / np.sqrt(20))
    assert np.abs(z).max() < 4.5, np.abs(z).max()
