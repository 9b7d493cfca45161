"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical
seeded inputs and identical Philox draws.

Tolerances: FP64 tracking must match every tally to 1e-10 (normwise: max |gpu - oracle| /
max |oracle|, per array); event counters are integers and must be equal. FP32 tracking
draws the same uniforms but walks in single precision: its steady temperature must match
the oracle's within 5e-4 of the wall-temperature span.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2506_09465_gb300 import workloads as WL  # noqa: E402
from gpu_helpers import gpu_solver, normwise_close, oracle_problem  # noqa: E402

RTOL64 = 1e-10


def cuda_T(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def cases():
    rng = np.random.default_rng(2024)
    out = []
    out.append(("1d_gray", [WL.random_instance(rng, 1, (37,), 1)], [1.0], [1.0]))
    out.append(("1d_nullcoll", [WL.Instance(1, (24,), (1.0,), np.where(np.arange(24) < 12, 10.0, 0.1)[None, :],
                                             np.array([1.0, -1.0]))], [1.0], [1.0]))
    out.append(("2d_gray_var", [WL.random_instance(rng, 2, (19, 13), 1, (0.02, 0.6))], [1.0], [1.0]))
    out.append(("2d_3band_src", [WL.random_instance(rng, 2, (11, 9), 3, (0.05, 2.0), source=True)],
                [0.5, 1.0, 1.5], [1.0, 0.7, 0.3]))
    out.append(("3d_gray", [WL.random_instance(rng, 3, (6, 5, 7), 1, (0.05, 0.5), source=True)], [1.0], [1.0]))
    return out


@pytest.mark.parametrize("name,insts,C,v", cases(), ids=[c[0] for c in cases()])
def test_sweep_fp64_matches_oracle(orc, name, insts, C, v):
    inst = insts[0]
    N, Nw = 60, 40
    rng = np.random.default_rng(7)
    T = rng.uniform(-0.5, 1.0, size=inst.ncells)
    p = oracle_problem(inst, C, v, N, Nw, seed=11)
    s = gpu_solver(inst, C, v, N, Nw, precision=0, tally=0, schedule=0, seed=11)
    assert s.layout.total_particles == int(p.n_band.sum()) * inst.ncells + int(p.n_wall_band.sum()) * sum(
        int(np.prod([inst.n[b] for b in range(inst.dim) if b != a])) * 2 for a in range(inst.dim))
    for epoch in (0, 5):
        r = orc.sweep(p, T, epoch)
        g = s.sweep(cuda_T(T), epoch)
        for key, ora in (("R", r.R), ("W", r.W), ("F", r.F), ("wall", r.wall)):
            ok, err = normwise_close(g[key].cpu().numpy(), ora, RTOL64)
            assert ok, (key, err)
        assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist()


@pytest.mark.parametrize("tally", [0, 1, 2])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_sweep_fp32_tracks_same_particles(orc, dim, tally):
    rng = np.random.default_rng(30 + dim)
    n = {1: (40,), 2: (16, 12), 3: (6, 6, 5)}[dim]
    inst = WL.random_instance(rng, dim, n, 1, (0.05, 0.8))
    N = 80
    T = rng.uniform(0.0, 1.0, size=inst.ncells)
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=3)
    r = orc.sweep(p, T, 0)
    s = gpu_solver(inst, [1.0], [1.0], N, N, precision=1, tally=tally, schedule=min(tally, 1), seed=3)
    g = s.sweep(cuda_T(T), 0)
    # Same draws; single-precision walks change a particle's cell only when it stops
    # within ~1e-7 of a face, so tallies agree to well below the statistical noise.
    for key, ora in (("R", r.R), ("W", r.W), ("F", r.F), ("wall", r.wall)):
        ok, err = normwise_close(g[key].cpu().numpy(), ora, 2e-3)
        assert ok, (key, err)
    c_g = g["counters"].cpu().numpy().astype(float)
    c_o = r.counters.astype(float)
    assert np.all(np.abs(c_g - c_o) <= 1e-3 * c_o + 2)


def test_macro_matches_oracle(orc):
    rng = np.random.default_rng(5)
    inst = WL.random_instance(rng, 2, (9, 7), 2, (0.1, 1.0))
    C, v = [0.7, 1.3], [1.0, 0.5]
    p = oracle_problem(inst, C, v, 30, 30)
    r = orc.sweep(p, rng.uniform(0, 1, inst.ncells), 0)
    Th, TE = orc.macro(p, r.R, r.W)
    s = gpu_solver(inst, C, v, 30, 30, precision=0)
    gTh, gTE = s.macro(cuda_T(r.R.ravel()), cuda_T(r.W.ravel()))
    assert np.allclose(gTh.cpu().numpy(), Th, rtol=1e-14, atol=0)
    assert np.allclose(gTE.cpu().numpy(), TE, rtol=1e-14, atol=0)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_newton_step_matches_direct_solve(orc, dim):
    rng = np.random.default_rng(40 + dim)
    n = {1: (30,), 2: (14, 11), 3: (6, 5, 4)}[dim]
    inst = WL.random_instance(rng, dim, n, 2, (0.01, 0.4))
    C, v = [1.0, 0.5], [1.0, 1.5]
    p = oracle_problem(inst, C, v, 40, 40)
    T = rng.uniform(0, 1, inst.ncells)
    r = orc.sweep(p, T, 0)
    Th, _ = orc.macro(p, r.R, r.W)
    T1, dT = orc.newton(p, T, Th, r.R)
    s = gpu_solver(inst, C, v, 40, 40, precision=0, cg_rtol=1e-14, cg_maxit=20000)
    gT = cuda_T(Th)
    it = s.newton_step(cuda_T(T), gT, cuda_T(r.R.ravel()))
    assert it > 0
    ok, err = normwise_close(gT.cpu().numpy() - Th, T1 - Th, 1e-9)
    assert ok, err


@pytest.mark.parametrize("rtol", [1e-3, 1e-5, 9.9e-6, 1e-11])
@pytest.mark.parametrize("dim,n,uniform", [(1, (30,), False), (2, (14, 11), False), (2, (160, 128), False),
                                           (3, (6, 5, 4), False), (1, (70,), True), (2, (48, 40), True),
                                           (2, (200, 7), True), (2, (150, 260), True)])
def test_correction_solve_meets_its_fp64_residual(orc, dim, n, uniform, rtol):
    # Separable operators (1D or 2D with uniform kappa) are solved by fast diagonalization;
    # the others by multigrid-preconditioned CG, with FP32 iterates from cg_rtol 1e-5 up (the
    # default 1e-3 among them) and FP64 iterates below. All of them refine in FP64: the
    # returned correction x meets ||s - A x|| <= cg_rtol ||s|| with A the oracle's FP64
    # operator and s its right-hand side (s = A dT of the oracle's direct banded solve), and
    # the solver reports its iterations (refinement passes for the direct solve).
    rng = np.random.default_rng(60 + dim)
    inst = WL.random_instance(rng, dim, n, 2, (0.01, 0.4))
    if uniform:  # the same tau in every cell of a band: uniform kappa
        inst.tau = np.repeat(rng.uniform(0.02, 0.4, size=(2, 1)), inst.ncells, axis=1)
    C, v = [1.0, 0.5], [1.0, 1.5]
    N = 40 if inst.ncells < 1000 else 4
    p = oracle_problem(inst, C, v, N, N)
    T = rng.uniform(0, 1, inst.ncells)
    r = orc.sweep(p, T, 0)
    Th, _ = orc.macro(p, r.R, r.W)
    T1, dT = orc.newton(p, T, Th, r.R)
    theta = orc.newton_theta(p)
    s = gpu_solver(inst, C, v, N, N, precision=0, cg_rtol=rtol)
    gT = cuda_T(Th)
    it = s.newton_step(cuda_T(T), gT, cuda_T(r.R.ravel()))
    assert it > 0
    x = (gT.cpu().numpy() - Th) / theta
    rhs = orc.diffusion_apply(p, dT / theta)  # the oracle returns the damped correction theta dT
    res = np.linalg.norm(rhs - orc.diffusion_apply(p, x)) / np.linalg.norm(rhs)
    assert res <= rtol * 1.001, res
    if uniform:
        assert it <= 6, it  # direct solve: a few refinement passes


def test_correction_solve_batch_mixes_solvers(orc):
    # One context whose instances take the three correction solvers in one launch: fast
    # diagonalization with every operand in shared memory (axes up to 128), the register-tiled
    # one (larger axes) and the multigrid PCG (varying kappa). Each instance's correction meets
    # its FP64 residual against the oracle's operator.
    rng = np.random.default_rng(64)
    insts = [WL.random_instance(rng, 2, n, 1, (0.02, 0.4)) for n in [(40, 30), (140, 135), (20, 18)]]
    for inst in insts[:2]:
        inst.tau = np.full_like(inst.tau, rng.uniform(0.05, 0.3))
    rtol = 1e-5
    N = 4
    s = gpu_solver(insts, [1.0], [1.0], N, N, precision=0, cg_rtol=rtol)
    ps = [oracle_problem(inst, [1.0], [1.0], N, N, instance=k) for k, inst in enumerate(insts)]
    Ts, Ths, Rs, dTs, thetas = [], [], [], [], []
    for k, (inst, p) in enumerate(zip(insts, ps)):
        T = rng.uniform(0, 1, inst.ncells)
        r = orc.sweep(p, T, 0)
        Th, _ = orc.macro(p, r.R, r.W)
        _, dT = orc.newton(p, T, Th, r.R)
        Ts.append(T)
        Ths.append(Th)
        Rs.append(r.R.ravel())
        dTs.append(dT)
        thetas.append(orc.newton_theta(p))
    gT = cuda_T(np.concatenate(Ths))
    s.newton_step(cuda_T(np.concatenate(Ts)), gT, cuda_T(np.concatenate(Rs)))
    got = gT.cpu().numpy()
    co = s.cell_off
    for k, p in enumerate(ps):
        x = (got[co[k]:co[k + 1]] - Ths[k]) / thetas[k]
        rhs = orc.diffusion_apply(p, dTs[k] / thetas[k])
        res = np.linalg.norm(rhs - orc.diffusion_apply(p, x)) / np.linalg.norm(rhs)
        assert res <= rtol * 1.001, (k, res)


@pytest.mark.parametrize("newton", [0, 1])
def test_steady_fp64_matches_oracle(orc, newton):
    inst = WL.slab(40, 0.1, 1.0, -1.0).instances[0]
    N = 200
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=1)
    T_o, it_o, res_o, _ = orc.solve_steady(p, np.zeros(40), 1e-12, 3000, frozen=True, newton=bool(newton), dT_ref=2.0)
    s = gpu_solver(inst, [1.0], [1.0], N, N, precision=0, tally=0, schedule=0, seed=1, newton=newton,
                   cg_rtol=1e-14, cg_maxit=20000)
    T_g, it_g, res_g = s.solve_steady(None, 1e-12, 3000)
    assert res_o <= 1e-12 and res_g <= 1e-12
    ok, err = normwise_close(T_g.cpu().numpy(), T_o, 1e-9)
    assert ok, err
    assert abs(it_g - it_o) <= 2


def test_steady_fp32_within_5e4_of_span(orc):
    # FP32 tracking, frozen draws: steady T within 5e-4 of dT (the accuracy target).
    inst = WL.cavity(24, 0.1).instances[0]
    N = 256
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=2)
    T_o, _, res_o, _ = orc.solve_steady(p, np.zeros(inst.ncells), 1e-9, 500, frozen=True, newton=True, dT_ref=1.0)
    for tally in (0, 1, 2):
        s = gpu_solver(inst, [1.0], [1.0], N, N, precision=1, tally=tally, seed=2)
        T_g, it, res = s.solve_steady(None, 1e-9, 500)
        assert np.abs(T_g.cpu().numpy() - T_o).max() <= 5e-4, tally


def test_batch_equals_standalone(orc):
    rng = np.random.default_rng(77)
    insts = [WL.random_instance(rng, 2, n, 1, (0.05, 0.5), source=(k % 2 == 0), L=(1.0, 1.0))
             for k, n in enumerate([(8, 8), (13, 5), (20, 17)])]
    N = 50
    Ts = [rng.uniform(0, 1, i.ncells) for i in insts]
    sb = gpu_solver(insts, [1.0], [1.0], N, N, precision=0, tally=0, instance_base=4, seed=9)
    gb = sb.sweep(cuda_T(np.concatenate(Ts)), 3)
    Rb = gb["R"].cpu().numpy()
    for k, inst in enumerate(insts):
        s1 = gpu_solver(inst, [1.0], [1.0], N, N, precision=0, tally=0, instance_base=4 + k, seed=9)
        g1 = s1.sweep(cuda_T(Ts[k]), 3)
        co = sb.cell_off
        ok, err = normwise_close(Rb[co[k]:co[k + 1]], g1["R"].cpu().numpy(), 1e-12)
        assert ok, (k, err)
        # and the oracle agrees with the standalone instance
        p = oracle_problem(inst, [1.0], [1.0], N, N, seed=9, instance=4 + k)
        ok, err = normwise_close(g1["R"].cpu().numpy(), orc.sweep(p, Ts[k], 3).R, RTOL64)
        assert ok, err


def test_adjoint_matches_dense_transpose(orc):
    rng = np.random.default_rng(8)
    inst = WL.random_instance(rng, 2, (6, 5), 1, (0.1, 0.8), source=True)
    N = 40
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=4)
    g = np.zeros(inst.ncells)
    g[[7, 8, 13, 14]] = 0.25
    gQ, gW, lam, A, Bw = orc.adjoint_dense(p, g)
    s = gpu_solver(inst, [1.0], [1.0], N, N, precision=0, tally=0, seed=4, cg_rtol=1e-14, cg_maxit=20000)
    gs, gw, gl = s.adjoint(cuda_T(g), tol=1e-13, max_iter=500)
    for got, ref in ((gl, lam), (gs, gQ), (gw, gW)):
        ok, err = normwise_close(got.cpu().numpy(), ref, 1e-9)
        assert ok, err


@pytest.mark.parametrize("fast,kn", [(False, 1.0), (True, 0.01), (True, 1.0), (True, 10.0)])
def test_full_size_cavity_sampled_emitters(orc, fast, kn):
    # The 128 x 128 cavity at the bench's particle count, with only a few cells hot (so the
    # oracle traces only their particles). Plain FP64 path: every tally agrees. Fast path in
    # the bench's launch configuration (pass-synchronous kernel, two-group face tallies in the
    # shared-memory window, FP64 replay of deferred flights): counters equal, R and W to
    # summation order, faces and walls within the window's fixed-point rounding (each
    # particle's weight rounded to 2^-26 of the largest).
    inst = WL.cavity(128, kn).instances[0]
    inst.wall_T = np.zeros(4)
    T = np.zeros(inst.ncells)
    T[[0, 5000, 8256, 16383]] = [1.0, 0.5, -0.25, 2.0]
    N = 1024
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=0)
    r = orc.sweep(p, T, 0)
    opt = {} if fast else dict(precision=0, tally=0, schedule=0)
    s = gpu_solver(inst, [1.0], [1.0], N, N, seed=0, **opt)
    g = s.sweep(cuda_T(T), 0)
    assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist()
    for key, ora in (("R", r.R), ("W", r.W), ("F", r.F), ("wall", r.wall)):
        ok, err = normwise_close(g[key].cpu().numpy(), ora, 1e-6 if fast and key in ("F", "wall") else RTOL64)
        assert ok, (key, err)


def test_full_size_conservation_every_mode():
    # Any size, any mode: the net inflow from the face tallies equals absorbed minus emitted
    # power in every cell, and walls balance globally.
    inst = WL.cavity(128, 0.1).instances[0]
    rng = np.random.default_rng(3)
    T = rng.uniform(0, 1, inst.ncells)
    for prec, tally, sched in ((0, 0, 0), (1, 0, 0), (1, 1, 1)):
        s = gpu_solver(inst, [1.0], [1.0], 1024, 1024, precision=prec, tally=tally, schedule=sched)
        g = s.sweep(cuda_T(T), 0)
        F = g["F"].cpu().numpy()
        R = g["R"].cpu().numpy()
        n = 128
        Fx = F[: (n + 1) * n].reshape(n, n + 1)
        Fy = F[(n + 1) * n:].reshape(n + 1, n)
        inflow = (Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]).ravel()
        V = 1.0 / n ** 2
        emitted = T * V / 0.1
        scale = np.abs(emitted).max()
        tol = 1e-9 if tally == 0 else 1e-4
        assert np.abs(inflow - (R - emitted)).max() <= tol * scale * 50, (prec, tally)
        wall_em = 1.0 / 4.0 * 1.0
        assert abs((g["wall"].cpu().numpy().sum() - wall_em) - (emitted.sum() - R.sum())) <= 1e-6 * emitted.sum()


def test_statistical_average_matches_oracle(orc):
    # Averaging after convergence (Sec. 4.4): 12 fresh-draw iterations from the converged
    # state; the FP64 path takes the oracle's draws and update, so the mean, the sample
    # variance of the iterates and the mean face power agree; the fast FP32 path's mean is
    # within 5e-4 of the wall span.
    inst = WL.cavity(24, 0.1).instances[0]
    N = 256
    p = oracle_problem(inst, [1.0], [1.0], N, N, seed=8)
    T0, _, _, _ = orc.solve_steady(p, np.zeros(inst.ncells), 1e-9, 300, frozen=True, newton=True, dT_ref=1.0)
    T_last, Tm, Tv, Fm = orc.average(p, T0, 12, 500)
    s = gpu_solver(inst, [1.0], [1.0], N, N, precision=0, tally=0, schedule=0, seed=8, cg_rtol=1e-12)
    T = cuda_T(T0)
    mean, var, F = s.average(T, 12, 500, want_F=True)
    for got, ref, tol in ((T, T_last, 1e-9), (mean, Tm, 1e-9), (F, Fm, 1e-9), (var, Tv, 1e-6)):
        ok, err = normwise_close(got.cpu().numpy(), ref, tol)
        assert ok, err
    assert np.all(Tv > 0)
    s32 = gpu_solver(inst, [1.0], [1.0], N, N, seed=8)
    m32, _, _ = s32.average(cuda_T(T0), 12, 500, want_var=False)
    assert np.abs(m32.cpu().numpy() - Tm).max() <= 5e-4


def test_compensated_fp32_tallies_match_fp64_tallies():
    # Same particles and FP32 walks, tallies either FP64 atomics or compensated FP32 pairs:
    # the two differ by rounding only (about n 2^-48 relative after n additions), far below
    # the FP32 walk's own effect; counters are identical. Includes a 200^2 instance whose
    # x-faces miss the shared-memory window, so face tallies take the compensated path too.
    wl = WL.cavity_sweep(64, (0.05, 1.0))
    wl.instances.append(WL.cavity(200, 0.3).instances[0])
    rng = np.random.default_rng(9)
    T = cuda_T(rng.uniform(0, 1, wl.total_cells))
    out = []
    for tally in (1, 2):
        s = gpu_solver(wl.instances, [1.0], [1.0], 256, 256, seed=6, tally=tally)
        out.append(s.sweep(T, 1))
    assert out[0]["counters"].cpu().tolist() == out[1]["counters"].cpu().tolist()
    for key in ("R", "W", "F", "wall"):
        ok, err = normwise_close(out[1][key].cpu().numpy(), out[0][key].cpu().numpy(), 1e-9)
        assert ok, (key, err)


def test_staged_tunables_change_speed_not_results():
    # refill threshold, particles per warp claim and crossings per walk phase only reorder
    # the work: the same particles take the same FP32 steps, so counters and the integer
    # x-face window are exact and R, W, F differ by FP64 atomic order alone.
    wl = WL.cavity_sweep(64, (0.05, 1.0))
    rng = np.random.default_rng(8)
    T = cuda_T(rng.uniform(0, 1, wl.total_cells))
    ref = None
    for kw in (dict(), dict(refill_lanes=4, warp_grab=128, walk_k=8), dict(refill_lanes=24, warp_grab=512, walk_k=32),
               dict(refill_lanes=16, warp_grab=32, walk_k=1)):
        s = gpu_solver(wl.instances, [1.0], [1.0], 512, 512, seed=4, **kw)
        g = s.sweep(T, 3)
        if ref is None:
            ref = g
            continue
        assert g["counters"].cpu().tolist() == ref["counters"].cpu().tolist(), kw
        for key in ("R", "W", "F", "wall"):
            ok, err = normwise_close(g[key].cpu().numpy(), ref[key].cpu().numpy(), 1e-12)
            assert ok, (kw, key, err)
    s = gpu_solver(wl.instances, [1.0], [1.0], 512, 512, seed=4)
    t = s.autotune(T, 3, allow_k32=True)
    assert t["refill_lanes"] in (0, 4, 8, 16, 24) and t["warp_grab"] in (128, 256, 512)
    assert t["walk_k"] in (8, 16, 32) and t["tally"] in (1, 2) and 0 < t["sweep_ms"] <= t["baseline_ms"]
    g = s.sweep(T, 3)
    assert g["counters"].cpu().tolist() == ref["counters"].cpu().tolist()
    ok, err = normwise_close(g["R"].cpu().numpy(), ref["R"].cpu().numpy(), 1e-9 if t["tally"] == 2 else 1e-12)
    assert ok, err
    with pytest.raises(Exception):
        gpu_solver(wl.instances, [1.0], [1.0], 512, 512, precision=0, tally=0, schedule=0).autotune(T)


def test_graph_replay_matches_plain_loop():
    # Frozen draws: the CUDA-graph replay (two iterations per replay) and the plain loop
    # run the same iteration; they differ only in atomic summation order.
    inst = WL.cavity(40, 0.1).instances[0]
    outs = []
    for graphs in (1, 0):
        s = gpu_solver(inst, [1.0], [1.0], 256, 256, use_graphs=graphs, seed=5)
        T, it, res = s.solve_steady(None, 1e-9, 200)
        assert res <= 1e-9
        outs.append((T.cpu().numpy(), it))
    ok, err = normwise_close(outs[0][0], outs[1][0], 1e-8)
    assert ok, err
    assert outs[0][1] >= outs[1][1] and outs[0][1] - outs[1][1] <= 1


@pytest.mark.parametrize("refill", [4, 16])
def test_pass_synchronous_adjoint_matches_per_lane_refill(refill):
    # The 2D adjoint re-trace runs pass by pass by default (refill_lanes 0) and with the
    # per-lane refill of the staged kernel otherwise: the same particles, draws and gathers,
    # so the adjoint fields and gradients agree to FP64 summation order; on a non-gray
    # (acceptance-tested) and a gray instance.
    rng = np.random.default_rng(23)
    insts = [WL.random_instance(rng, 2, (24, 20), 2, (0.05, 0.6), source=True), WL.cavity(32, 0.3).instances[0]]
    for inst in insts:
        g = np.zeros(inst.ncells)
        g[[40, 41, 70, 71, 100]] = 0.2
        out = []
        for rl in (0, refill):
            C, v = ([1.0, 0.5], [1.0, 1.5]) if inst.tau.shape[0] == 2 else ([1.0], [1.0])
            s = gpu_solver(inst, C, v, 64, 64, seed=9, cg_rtol=1e-12, refill_lanes=rl)
            out.append([x.cpu().numpy() for x in s.adjoint(cuda_T(g), tol=1e-11, max_iter=500)])
        for a_, b_ in zip(out[0], out[1]):
            ok, err = normwise_close(a_, b_, 1e-9)
            assert ok, err


def test_adjoint_gradient_exact_for_frozen_map():
    # With draws fixed the steady state is affine in theta = (Q, T_w) (T_ref = 0), so
    # J = g . T* satisfies J = sum_k theta_k dJ/dtheta_k and central differences equal the
    # adjoint gradient up to rounding and solver tolerances. Also through the autograd
    # Function.
    from paper_2506_09465_gb300.solver import IugkpSteady
    rng = np.random.default_rng(21)
    inst = WL.random_instance(rng, 2, (12, 10), 1, (0.05, 0.5), source=True)
    N = 64
    s = gpu_solver(inst, [1.0], [1.0], N, N, seed=2, cg_rtol=1e-12)
    Q = torch.as_tensor(inst.source, device="cuda")
    Tw = torch.as_tensor(inst.wall_T, device="cuda")
    g = torch.zeros(inst.ncells, dtype=torch.float64, device="cuda")
    g[[30, 31, 42, 43]] = 0.25

    def J(Qv, Twv):
        s.set_source(Qv)
        s.set_wall_T(Twv)
        T, it, res = s.solve_steady(None, 1e-13, 500)
        return float((g * T).sum())

    J0 = J(Q, Tw)
    s.set_source(Q)
    s.set_wall_T(Tw)
    gs, gw, _ = s.adjoint(g, tol=1e-13, max_iter=500)
    euler = float((Q * gs).sum() + (Tw * gw).sum())
    assert abs(euler - J0) < 1e-9 * abs(J0)
    h = 1e-3
    for i in (31, 55):
        e = torch.zeros_like(Q)
        e[i] = h
        fd = (J(Q + e, Tw) - J(Q - e, Tw)) / (2 * h)
        assert abs(fd - float(gs[i])) < 1e-7 * max(1.0, abs(float(gs[i])))
    e = torch.zeros_like(Tw)
    e[3] = h
    fd = (J(Q, Tw + e) - J(Q, Tw - e)) / (2 * h)
    assert abs(fd - float(gw[3])) < 1e-7
    # autograd
    Qr = Q.clone().requires_grad_(True)
    Twr = Tw.clone().requires_grad_(True)
    T = IugkpSteady.apply(Qr, Twr, s, 1e-13, 500)
    (g * T).sum().backward()
    assert torch.allclose(Qr.grad, gs, rtol=1e-9, atol=1e-12)
    assert torch.allclose(Twr.grad, gw, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("n", [96, 180])
def test_two_group_face_tallies_match_plain_fp64_faces(n):
    # 2D instances whose faces all fit the shared-memory window split the particles by the
    # axis they cross less often: each group tallies only those faces and the rest follow
    # from the group's own power balance (n = 96). At n = 180 only the faces normal to x fit:
    # every particle tallies those and the faces normal to y follow from conservation. Both
    # run the pass-synchronous kernel. Against the plain FP64 sweep of the same particles
    # (every face tallied by FP64 atomics), on every face kind (interior, each wall) with
    # hot, cold and negative wall temperatures: a difference is a particle whose FP32 walk
    # ended within rounding of a face (a tie), so every face, cell and wall differs by at
    # most a few particle weights, and only a small fraction differs at all.
    N, tau = 256, 0.5
    inst = WL.cavity(n, tau).instances[0]
    inst.wall_T = np.array([0.4, -0.3, 0.8, 1.0])
    rng = np.random.default_rng(21)
    T = rng.uniform(-0.2, 1.0, inst.ncells)
    h = 1.0 / n
    wmax = max(np.abs(T).max() * h * h / tau / N, np.abs(inst.wall_T).max() * h / 4.0 / N)
    out = []
    for prec, tally, sched in ((0, 0, 0), (1, 1, 1), (1, 2, 1)):
        s = gpu_solver(inst, [1.0], [1.0], N, N, precision=prec, tally=tally, schedule=sched, seed=12)
        out.append(s.sweep(cuda_T(T), 0))
    ref = {key: out[0][key].cpu().numpy() for key in ("R", "W", "F", "wall")}
    nx = (n + 1) * n
    kinds = {"x low wall": np.s_[0:nx:n + 1], "x high wall": np.s_[n:nx:n + 1], "y low wall": np.s_[nx:nx + n],
             "y high wall": np.s_[nx + n * n:], "all": np.s_[:]}
    for g in out[1:]:
        c_g, c_0 = (np.array(x["counters"].cpu().tolist(), dtype=float) for x in (g, out[0]))
        assert c_g[0] == c_0[0] and np.all(np.abs(c_g - c_0) <= 1e-4 * c_0 + 5)
        for key, bound in (("R", 4 * wmax), ("W", 4 * wmax * tau), ("F", 4 * wmax), ("wall", 20 * wmax)):
            d = np.abs(g[key].cpu().numpy() - ref[key])
            assert d.max() <= bound, (key, d.max() / wmax)
            if key in ("R", "F"):
                assert np.mean(d > 0.01 * wmax) < 0.02, (key, np.mean(d > 0.01 * wmax))
        F = g["F"].cpu().numpy()
        for name, sl in kinds.items():
            assert np.abs(F[sl] - ref["F"][sl]).max() <= 4 * wmax, name
            assert np.abs(ref["F"][sl]).max() > 50 * wmax, name  # the faces carry real flux


@pytest.mark.parametrize("tally", [0, 1])
def test_set_tau_equals_fresh_context(orc, tally):
    # iugkp_set_field(TAU) on a context (two bands, source, per-face wall temperatures) gives
    # the sweep, macro update and Newton step of a context created with the new tau, and the
    # oracle's tallies for it (FP64 walk) at 1e-10.
    rng = np.random.default_rng(91)
    inst = WL.random_instance(rng, 2, (13, 9), 2, (0.05, 0.6), source=True)
    tau2 = rng.uniform(0.02, 0.9, size=inst.tau.shape)
    C, v = [1.0, 0.6], [1.0, 1.4]
    N = 48
    faceT = rng.uniform(-0.5, 1.0, size=2 * (13 + 9))
    kw = dict(precision=0 if tally == 0 else 1, tally=tally, schedule=0 if tally == 0 else 1, seed=4)
    s = gpu_solver(inst, C, v, N, N, **kw)
    s.set_wall_face_T(faceT)
    s.set_tau(tau2)
    inst2 = WL.Instance(inst.dim, inst.n, inst.L, tau2, inst.wall_T, inst.source, wall_face_T=faceT)
    f = gpu_solver(inst2, C, v, N, N, **kw)
    assert s.layout.total_particles == f.layout.total_particles
    T = cuda_T(rng.uniform(0.0, 1.0, inst.ncells))
    gs, gf = s.sweep(T, 2), f.sweep(T, 2)
    assert gs["counters"].cpu().tolist() == gf["counters"].cpu().tolist()
    for key in ("R", "W", "F", "wall"):
        ok, err = normwise_close(gs[key].cpu().numpy(), gf[key].cpu().numpy(), 1e-12)
        assert ok, (key, err)
    Ts, _ = s.macro(gs["R"])
    Tf, _ = f.macro(gf["R"])
    s.newton_step(T, Ts, gs["R"])
    f.newton_step(T, Tf, gf["R"])
    ok, err = normwise_close(Ts.cpu().numpy(), Tf.cpu().numpy(), 1e-12)
    assert ok, err
    if tally == 0:
        p = oracle_problem(inst2, C, v, N, N, seed=4)
        r = orc.sweep(p, T.cpu().numpy(), 2)
        ok, err = normwise_close(gs["R"].cpu().numpy(), r.R, RTOL64)
        assert ok, err
