"""Full-size GPU checks of the larger configurations (non-gray square, batch of 3D boxes,
non-gray adjoint batch). The oracle is compared on sampled emitters (only a few cells carry
power, so it traces only their particles) and on the smallest members; properties that
hold at any size (per-cell conservation, batch = standalone, exactness of the frozen-draw
adjoint) are checked on the whole workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_09465_gb300 import workloads as WL  # noqa: E402
from gpu_helpers import gpu_solver, normwise_close, oracle_problem  # noqa: E402


def cuda(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def inflow_2d(F, n0, n1, off=0):
    Fx = F[off: off + (n0 + 1) * n1].reshape(n1, n0 + 1)
    Fy = F[off + (n0 + 1) * n1: off + (n0 + 1) * n1 + n0 * (n1 + 1)].reshape(n1 + 1, n0)
    return (Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]).ravel()


def inflow_3d(F, n, off=0):
    n0 = n1 = n2 = n
    nx = (n0 + 1) * n1 * n2
    ny = n0 * (n1 + 1) * n2
    Fx = F[off: off + nx].reshape(n2, n1, n0 + 1)
    Fy = F[off + nx: off + nx + ny].reshape(n2, n1 + 1, n0)
    Fz = F[off + nx + ny: off + nx + ny + n0 * n1 * (n2 + 1)].reshape(n2 + 1, n1, n0)
    return (Fx[:, :, :-1] - Fx[:, :, 1:] + Fy[:, :-1, :] - Fy[:, 1:, :] + Fz[:-1] - Fz[1:]).ravel()


def test_nongray_square_sampled_emitters_match_oracle(orc):
    # 256 x 256, 80 band-branches, 1024 particles per cell: only three cells carry source.
    wl = WL.nongray_square(256, 40, 1024)
    inst = wl.instances[0]
    src = np.zeros(inst.ncells)
    src[[5000, 32896, 60000]] = [1.0, 2.0, 0.5]
    inst.source = src
    p = oracle_problem(inst, wl.C, wl.v, 1024, 1024, seed=0)
    r = orc.sweep(p, np.zeros(inst.ncells), 0)
    s = gpu_solver(inst, wl.C, wl.v, 1024, 1024, precision=0, tally=0, schedule=0, seed=0)
    assert s.layout.total_particles == int(p.n_band.sum()) * inst.ncells + int(p.n_wall_band.sum()) * 4 * 256
    g = s.sweep(cuda(np.zeros(inst.ncells)), 0)
    for key, ora in (("R", r.R), ("W", r.W), ("F", r.F), ("wall", r.wall)):
        ok, err = normwise_close(g[key].cpu().numpy(), ora, 1e-10)
        assert ok, (key, err)
    assert g["counters"].cpu().numpy().tolist() == r.counters.astype(np.int64).tolist()


def test_nongray_square_full_sweep_conserves():
    # Every cell emits (T = 0.2 plus the Gaussian source); fast path without the shared
    # x-face window (the instance's x-faces exceed it): per-cell balance and wall balance.
    wl = WL.nongray_square(256, 40, 1024)
    inst = wl.instances[0]
    s = gpu_solver(inst, wl.C, wl.v, 1024, 1024)
    T = np.full(inst.ncells, 0.2)
    g = s.sweep(cuda(T), 0)
    R = g["R"].cpu().numpy().reshape(len(wl.C), -1)
    V = 1.0 / 256 ** 2
    m = (wl.C[:, None] / inst.tau).sum(0)
    emitted = V * m * (T + inst.source / m)
    inflow = inflow_2d(g["F"].cpu().numpy(), 256, 256)
    scale = np.abs(emitted).max()
    assert np.abs(inflow - (R.sum(0) - emitted)).max() < 1e-8 * scale
    assert abs(g["wall"].cpu().numpy().sum() - (emitted.sum() - R.sum())) < 1e-8 * emitted.sum()
    c = g["counters"].cpu().numpy()
    assert c[0] == c[2] + c[4] and c[5] == 0


def test_box_batch_conserves_and_matches_standalone(orc):
    # 16 uneven 3D boxes (16^3 .. 64^3, 1.44 M cells), 256 particles per cell, source only.
    wl = WL.box_batch(16)
    s = gpu_solver(wl.instances, wl.C, wl.v, 256, 256, seed=7, instance_base=100)
    T = np.zeros(wl.total_cells)
    g = s.sweep(cuda(T), 0)
    F = g["F"].cpu().numpy()
    R = g["R"].cpu().numpy()
    for k in (0, 7, 15):
        inst = wl.instances[k]
        n = inst.n[0]
        co, fo = s.cell_off[k], s.face_off[k]
        V = 1.0 / n ** 3
        emitted = V * inst.source
        inflow = inflow_3d(F, n, fo)
        assert np.abs(inflow - (R[co:co + inst.ncells] - emitted)).max() < 1e-8 * emitted.max(), k
    # smallest box: batched FP64 sweep = oracle on the same instance id
    s64 = gpu_solver(wl.instances, wl.C, wl.v, 256, 256, seed=7, instance_base=100, precision=0, tally=0,
                     schedule=0)
    g64 = s64.sweep(cuda(T), 0)
    inst = wl.instances[0]
    p = oracle_problem(inst, wl.C, wl.v, 256, 256, seed=7, instance=100)
    r = orc.sweep(p, np.zeros(inst.ncells), 0)
    ok, err = normwise_close(g64["R"].cpu().numpy()[: inst.ncells], r.R, 1e-10)
    assert ok, err
    ok, err = normwise_close(g64["F"].cpu().numpy()[: s64.face_off[1]], r.F, 1e-10)
    assert ok, err


def test_box_batch_compensated_fp32_tallies_against_fp64():
    # The 16-box batch with compensated FP32 tallies against FP64 tallies (same particles):
    # equal counters, tallies within rounding, and the steady state of the smallest box
    # within 5e-4 of its span of the FP64-tally solve.
    wl = WL.box_batch(16)
    T = torch.zeros(wl.total_cells, dtype=torch.float64, device="cuda")
    g = []
    for tally in (1, 2):
        s = gpu_solver(wl.instances, wl.C, wl.v, 256, 256, seed=7, instance_base=100, tally=tally)
        g.append(s.sweep(T, 0))
    assert g[0]["counters"].cpu().tolist() == g[1]["counters"].cpu().tolist()
    for key in ("R", "W", "F", "wall"):
        ok, err = normwise_close(g[1][key].cpu().numpy(), g[0][key].cpu().numpy(), 1e-9)
        assert ok, (key, err)
    small = [wl.instances[0], wl.instances[3]]
    Ts = []
    for tally in (1, 2):
        s = gpu_solver(small, wl.C, wl.v, 256, 256, seed=7, tally=tally)
        Tt, it, res = s.solve_steady(None, 1e-8, 300)
        assert res <= 1e-8
        Ts.append(Tt.cpu().numpy())
    span = Ts[0].max() - Ts[0].min()
    assert np.abs(Ts[1] - Ts[0]).max() <= 5e-4 * span


def test_nongray_adjoint_dense_transpose_8x8(orc):
    # 8 x 8, 40 band-branches: re-trace adjoint (FP64) = dense transpose of the oracle map.
    C, v, tb, _ = WL.silicon_like_bands(20)
    nc = 64
    rng = np.random.default_rng(3)
    tau = np.repeat(tb[:, None], nc, axis=1) * rng.uniform(0.8, 1.2, size=(len(C), nc))
    inst = WL.Instance(2, (8, 8), (1.0, 1.0), tau, np.array([0.0, 0.3, 0.0, 1.0]), rng.uniform(0, 1, nc))
    p = oracle_problem(inst, C, v, 128, 128, seed=1)
    g = WL.hotspot_objective(inst, 0.1)
    gQ, gW, lam, A, Bw = orc.adjoint_dense(p, g)
    s = gpu_solver(inst, C, v, 128, 128, precision=0, tally=0, schedule=0, seed=1, cg_rtol=1e-13, cg_maxit=20000)
    gs, gw, gl = s.adjoint(cuda(g), tol=1e-13, max_iter=1000)
    for got, ref in ((gl, lam), (gs, gQ), (gw, gW)):
        ok, err = normwise_close(got.cpu().numpy(), ref, 1e-8)
        assert ok, err


def test_nongray_batch_adjoint_fd_and_euler():
    # Four members of the non-gray adjoint batch (64^2 .. 128^2, 40 band-branches), fast
    # path: J = mean T over each hotspot; central differences (h = 1e-3) on two source cells
    # and a wall, and the Euler identity J = sum theta dJ/dtheta.
    wl = WL.nongray_batch(4, 64, 128, 20, 128)
    s = gpu_solver(wl.instances, wl.C, wl.v, 128, 128, seed=11, cg_rtol=1e-12)
    g = np.concatenate([WL.hotspot_objective(i, 0.1) for i in wl.instances])
    gt = cuda(g)
    Q = cuda(np.concatenate([i.source for i in wl.instances]))
    Tw = cuda(np.concatenate([i.wall_T for i in wl.instances]))

    def J(Qv, Twv):
        s.set_source(Qv)
        s.set_wall_T(Twv)
        T, it, res = s.solve_steady(None, 1e-12, 400)
        return float((gt * T).sum())

    J0 = J(Q, Tw)
    s.set_source(Q)
    s.set_wall_T(Tw)
    gs, gw, _ = s.adjoint(gt, tol=1e-12, max_iter=400)
    euler = float((Q * gs).sum() + (Tw * gw).sum())
    assert abs(euler - J0) < 1e-8 * abs(J0)
    h = 1e-3
    co = s.cell_off
    for i in (co[1] + 64 * 40 + 40, co[3] + 10):
        e = torch.zeros_like(Q)
        e[i] = h
        fd = (J(Q + e, Tw) - J(Q - e, Tw)) / (2 * h)
        assert abs(fd - float(gs[i])) < 1e-5 * abs(float(gs[i])) + 1e-9
    e = torch.zeros_like(Tw)
    e[5] = h
    fd = (J(Q, Tw + e) - J(Q, Tw - e)) / (2 * h)
    assert abs(fd - float(gw[5])) < 1e-5 * abs(float(gw[5])) + 1e-9
