"""Pins for the oracle's macro-prediction (inexact Newton) step, steady driver and
adjoint (arXiv 2506.09465 Sec. 3.3, Eqs. "macro-q-eqn" .. "linear-q"; Sec. 2 Eq. "sum-g"
makes a frozen-draw sweep an affine map, whose transpose the adjoint applies).
"""
import numpy as np
import pytest


def prob(orc, dim, n, L, tau, wall_T, N=100, C=(1.0,), v=(1.0,), source=None, seed=0):
    nc = int(np.prod(n))
    tau = np.asarray(tau, dtype=np.float64)
    if tau.ndim <= 1:
        tau = np.broadcast_to(tau, (nc,)).reshape(1, nc)
    return orc.Problem(dim, n, L, np.asarray(C, float), np.asarray(v, float), tau, np.asarray(wall_T, float),
                       np.full(len(C), N), np.full(len(C), N), source=source, seed=seed)


def test_diffusion_stencil_exact_on_quadratics(orc):
    n = 16
    p = prob(orc, 1, (n,), (1.0,), 0.3, [0, 0])
    kappa = 0.3 / 3.0
    x = (np.arange(n) + 0.5) / n
    y = orc.diffusion_apply(p, x * (1 - x))
    assert np.allclose(y[1:-1], 2.0 * kappa, rtol=1e-12)   # -kappa T'' with T'' = -2


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_diffusion_operator_symmetric_and_solver_inverts(orc, dim):
    n = {1: (13,), 2: (7, 5), 3: (4, 3, 5)}[dim]
    L = {1: (1.0,), 2: (1.0, 0.6), 3: (1.0, 0.6, 1.3)}[dim]
    rng = np.random.default_rng(10 + dim)
    nc = int(np.prod(n))
    p = orc.Problem(dim, n, L, np.array([1.0, 2.0]), np.array([1.0, 0.3]), rng.uniform(0.01, 1.0, (2, nc)),
                    np.zeros(2 * dim), np.array([1, 1]), np.array([1, 1]))
    a, b = rng.normal(size=nc), rng.normal(size=nc)
    Aa, Ab = orc.diffusion_apply(p, a), orc.diffusion_apply(p, b)
    assert abs(a @ Ab - b @ Aa) < 1e-12 * np.abs(Aa).sum()
    assert a @ Aa > 0
    assert np.allclose(orc.diffusion_solve(p, Aa), a, rtol=1e-9, atol=1e-10)


def test_diffusion_solve_converges_to_continuum_second_order(orc):
    # 1D: -kappa u'' = f with the vacuum (Marshak) wall condition kappa |u'| = (C v / 2) u
    # has u = f x (1 - x) / (2 kappa) + f / (C v); the finite-volume solution converges
    # at second order.
    f, tau = 1.0, 0.3
    kappa = tau / 3.0
    errs = []
    for n in (8, 16, 32):
        p = prob(orc, 1, (n,), (1.0,), tau, [0, 0])
        x = (np.arange(n) + 0.5) / n
        u = f * x * (1 - x) / (2 * kappa) + f / 1.0
        sol = orc.diffusion_solve(p, np.full(n, f))
        errs.append(np.abs(sol - u).max())
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0
    assert errs[2] < 2e-3 * u.max()


def test_diffusion_wall_conductance_limits(orc):
    # Optically thin wall cell: the vacuum condition dominates (flux -> C v T / 2);
    # thick: half-cell conduction dominates (flux -> 2 kappa T / h).
    for tau, expect in ((1e3, lambda k, h: 0.5 / h), (1e-4, lambda k, h: 2 * k / h / h)):
        n = 4
        p = prob(orc, 1, (n,), (1.0,), tau, [0, 0])
        e = np.zeros(n)
        e[0] = 1.0
        y = orc.diffusion_apply(p, e)
        k, h = tau / 3.0, 1.0 / n
        interior = k / h / h
        assert abs((y[0] - interior) / expect(k, h) - 1.0) < 0.02


def test_newton_leaves_fixed_point_unchanged(orc):
    n = 20
    p = prob(orc, 1, (n,), (1.0,), 0.3, [1.0, -1.0], N=200)
    T0 = np.zeros(n)
    Tp, itp, resp, _ = orc.solve_steady(p, T0, 1e-12, 2000, frozen=True, newton=False, dT_ref=2.0)
    Tn, itn, resn, _ = orc.solve_steady(p, T0, 1e-12, 2000, frozen=True, newton=True, dT_ref=2.0)
    assert resp <= 1e-12 and resn <= 1e-12
    assert np.allclose(Tp, Tn, atol=1e-9)
    assert itn < itp


@pytest.mark.parametrize("n", [25, 100])
def test_newton_accelerates_small_knudsen(orc, n):
    # Kn = 0.01 (cells of optical thickness 4 and 1): plain iteration contracts very
    # slowly (Table 1 trend); the damped diffusion correction converges in a few dozen.
    # The frozen-draw map must resolve the slow diffusive mode: its statistical error on
    # that mode (~ pi lambda / sqrt(N_total)) has to stay below its decay rate
    # (~ pi^2 lambda^2 / 3), hence 1000 particles per cell here.
    p = prob(orc, 1, (n,), (1.0,), 0.01, [1.0, 0.0], N=1000)
    T0 = np.zeros(n)
    _, itn, resn, hn = orc.solve_steady(p, T0, 1e-8, 200, frozen=True, newton=True, dT_ref=1.0)
    _, itp, resp, hp = orc.solve_steady(p, T0, 1e-8, itn * 10, frozen=True, newton=False, dT_ref=1.0)
    assert resn <= 1e-8 and itn <= 60
    assert resp > 1e-8            # plain has not converged in 10x the iterations


def test_newton_step_matches_definition(orc):
    n = (5, 4)
    rng = np.random.default_rng(5)
    p = prob(orc, 2, n, (1.0, 0.8), rng.uniform(0.05, 0.5, 20), [0.3, 0.0, 0.0, 1.0], N=50)
    T = rng.uniform(0, 1, 20)
    r = orc.sweep(p, T, 0)
    Th, _ = orc.macro(p, r.R, r.W)
    T1, dT = orc.newton(p, T, Th, r.R)
    V = p.volume()
    m = orc.cell_m(p)
    s = (r.R.sum(0) - m * T * V) / V
    theta = orc.newton_theta(p)
    assert 0.0 < theta <= 1.0
    assert np.allclose(orc.diffusion_apply(p, dT), theta * s, rtol=1e-9, atol=1e-12)
    assert np.allclose(T1, Th + dT, rtol=1e-15)
    assert np.allclose(s, m * (Th - T), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_adjoint_retrace_is_dense_transpose(orc, dim):
    n = {1: (6,), 2: (3, 3)}[dim]
    L = {1: (1.0,), 2: (1.0, 1.0)}[dim]
    nc = int(np.prod(n))
    rng = np.random.default_rng(20 + dim)
    p = orc.Problem(dim, n, L, np.array([1.0, 0.5]), np.array([1.0, 2.0]), rng.uniform(0.1, 1.0, (2, nc)),
                    np.zeros(2 * dim), np.array([30, 20]), np.array([25, 15]))
    A, Bw = orc.assemble_affine(p, 4)
    lam = rng.normal(size=nc)
    at, gw = orc.adjoint_apply(p, lam, 4)
    assert np.allclose(at, A.T @ lam, rtol=1e-11, atol=1e-13)
    assert np.allclose(gw, Bw.T @ lam, rtol=1e-11, atol=1e-13)


def test_adjoint_gradient_euler_identity_and_fd(orc):
    # J(theta) = g . T*(theta) is linear in theta = (Q, T_w) (T_ref = 0), so
    # J = sum_k theta_k dJ/dtheta_k, and central differences are exact up to rounding.
    n = (3, 3)
    nc = 9
    rng = np.random.default_rng(7)
    tau = rng.uniform(0.2, 1.0, nc)
    Q = rng.uniform(0.0, 2.0, nc)
    Tw = np.array([0.3, 0.0, 0.5, 1.0])
    g = np.zeros(nc)
    g[[4, 5]] = 0.5
    p = prob(orc, 2, n, (1.0, 1.0), tau, Tw, N=60, source=Q)

    def J(Qv, Twv):
        q = prob(orc, 2, n, (1.0, 1.0), tau, Twv, N=60, source=Qv)
        T, it, res, _ = orc.solve_steady(q, np.zeros(nc), 1e-14, 2000, frozen=True, newton=True, dT_ref=1.0)
        return g @ T

    gQ, gW, lam, A, Bw = orc.adjoint_dense(p, g)
    J0 = J(Q, Tw)
    assert abs(J0 - (Q @ gQ + Tw @ gW)) < 1e-10 * abs(J0)
    h = 1e-3
    for i in (0, 4):
        e = np.zeros(nc)
        e[i] = h
        fd = (J(Q + e, Tw) - J(Q - e, Tw)) / (2 * h)
        assert abs(fd - gQ[i]) < 1e-8 * max(1.0, abs(gQ[i]))
    e = np.zeros(4)
    e[3] = h
    fd = (J(Q, Tw + e) - J(Q, Tw - e)) / (2 * h)
    assert abs(fd - gW[3]) < 1e-8
    gQ2, gW2, lam2, it = orc.adjoint_iterative(p, g, tol=1e-13)
    assert np.allclose(lam2, lam, rtol=1e-10, atol=1e-12)
    assert np.allclose(gQ2, gQ, rtol=1e-9, atol=1e-12)
    assert np.allclose(gW2, gW, rtol=1e-9, atol=1e-12)
