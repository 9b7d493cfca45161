"""Degenerate shapes and fields on the GPU against the oracle (Sec. 3.1 steps (1)-(3), Sec. 3.2
candidates): single-cell, single-row, single-column and single-layer grids, one particle per
cell and per wall face, a zero field (every particle weighs zero), and a ragged batch (a 1 x 1
instance beside a 13 x 7 one, each with its own Philox instance id). The plain FP64 path must
match every tally to 1e-10 with equal counters; the fast path (FP32 walk with FP64 decisions,
staged tallies) must have equal counters and R equal to summation order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_09465_gb300 import workloads as WL  # noqa: E402
from gpu_helpers import gpu_solver, normwise_close, oracle_problem  # noqa: E402

SHAPES = [(1, (1,)), (1, (2,)), (2, (9, 1)), (2, (1, 7)), (2, (1, 1)), (3, (5, 4, 1)), (3, (1, 1, 3)),
          (3, (1, 1, 1))]


def cuda_T(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def shape_case(dim, n, seed):
    rng = np.random.default_rng(seed)
    inst = WL.random_instance(rng, dim, n, 1, (0.05, 0.8), source=True)
    T = rng.uniform(-0.3, 1.0, size=inst.ncells)
    return inst, T


def check_plain(orc, inst, T, N, Nw, seed, instance_base=0):
    p = oracle_problem(inst, [1.0], [1.0], N, Nw, seed=seed, instance=instance_base)
    s = gpu_solver(inst, [1.0], [1.0], N, Nw, seed=seed, instance_base=instance_base, precision=0, tally=0,
                   schedule=0)
    for epoch in (0, 5):
        r = orc.sweep(p, T, epoch)
        g = s.sweep(cuda_T(T), epoch)
        assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist(), epoch
        for key, ora in (("R", r.R), ("W", r.W), ("F", r.F), ("wall", r.wall)):
            ok, err = normwise_close(g[key].cpu().numpy(), ora, 1e-10)
            assert ok, (epoch, key, err)


def check_fast(orc, inst, T, N, Nw, seed, tally):
    p = oracle_problem(inst, [1.0], [1.0], N, Nw, seed=seed)
    s = gpu_solver(inst, [1.0], [1.0], N, Nw, seed=seed, precision=1, tally=tally)
    for epoch in (0, 5):
        r = orc.sweep(p, T, epoch)
        g = s.sweep(cuda_T(T), epoch)
        assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist(), epoch
        ok, err = normwise_close(g["R"].cpu().numpy(), r.R, 1e-10 if tally == 1 else 1e-9)
        assert ok, (epoch, "R", err)
        for key, ora in (("W", r.W), ("F", r.F), ("wall", r.wall)):
            ok, err = normwise_close(g[key].cpu().numpy(), ora, 2e-3)
            assert ok, (epoch, key, err)


@pytest.mark.parametrize("dim,n", SHAPES, ids=["x".join(map(str, n)) for _, n in SHAPES])
def test_degenerate_shapes_plain_fp64_match_oracle(orc, dim, n):
    inst, T = shape_case(dim, n, 100 + len(n) + sum(n))
    check_plain(orc, inst, T, 96, 64, seed=4)


@pytest.mark.parametrize("tally", [1, 2])
@pytest.mark.parametrize("dim,n", SHAPES, ids=["x".join(map(str, n)) for _, n in SHAPES])
def test_degenerate_shapes_fast_path_take_the_fp64_decisions(orc, dim, n, tally):
    inst, T = shape_case(dim, n, 200 + len(n) + sum(n))
    check_fast(orc, inst, T, 96, 64, seed=5, tally=tally)


@pytest.mark.parametrize("dim,n", [(1, (7,)), (2, (6, 5)), (3, (3, 4, 2))])
def test_one_particle_per_cell_and_wall_face(orc, dim, n):
    inst, T = shape_case(dim, n, 300 + dim)
    check_plain(orc, inst, T, 1, 1, seed=6)
    check_fast(orc, inst, T, 1, 1, seed=6, tally=1)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_field_gives_zero_tallies(orc, precision):
    # T = 0 everywhere, walls at 0, no source: every particle weighs zero, so every tally is
    # exactly zero on both sides and the counters agree.
    inst = WL.Instance(2, (8, 6), (1.0, 0.7), np.random.default_rng(7).uniform(0.05, 0.8, size=(1, 48)),
                       np.zeros(4))
    T = np.zeros(inst.ncells)
    p = oracle_problem(inst, [1.0], [1.0], 32, 32, seed=2)
    opt = dict(precision=0, tally=0, schedule=0) if precision == 0 else dict(precision=1, tally=1)
    s = gpu_solver(inst, [1.0], [1.0], 32, 32, seed=2, **opt)
    r = orc.sweep(p, T, 0)
    g = s.sweep(cuda_T(T), 0)
    for key in ("R", "W", "F", "wall"):
        assert np.all(g[key].cpu().numpy() == 0.0), key
    assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist()


@pytest.mark.parametrize("fast", [False, True])
def test_ragged_batch_matches_each_instance(orc, fast):
    # A 1 x 1 instance and a 13 x 7 one in one context: instance k draws with Philox instance
    # id k, so each instance's tallies equal the oracle's run of that instance with that id.
    rng = np.random.default_rng(8)
    insts = [WL.random_instance(rng, 2, (1, 1), 1, (0.05, 0.8), source=True),
             WL.random_instance(rng, 2, (13, 7), 1, (0.05, 0.8), source=True)]
    Ts = [rng.uniform(-0.3, 1.0, size=i.ncells) for i in insts]
    opt = dict(precision=1, tally=1) if fast else dict(precision=0, tally=0, schedule=0)
    s = gpu_solver(insts, [1.0], [1.0], 64, 48, seed=9, **opt)
    g = s.sweep(cuda_T(np.concatenate(Ts)), 0)
    R, F = g["R"].cpu().numpy().ravel(), g["F"].cpu().numpy().ravel()
    c0 = f0 = 0
    for k, (inst, T) in enumerate(zip(insts, Ts)):
        p = oracle_problem(inst, [1.0], [1.0], 64, 48, seed=9, instance=k)
        r = orc.sweep(p, T, 0)
        nf = r.F.size
        ok, err = normwise_close(R[c0:c0 + inst.ncells], r.R.ravel(), 1e-10)
        assert ok, (k, "R", err)
        ok, err = normwise_close(F[f0:f0 + nf], r.F, 1e-10 if not fast else 2e-3)
        assert ok, (k, "F", err)
        c0 += inst.ncells
        f0 += nf
