"""Pins for the FP64 oracle against what the paper and the mathematics fix.

* Monte Carlo sweep means against the closed-form E_3 slab operator (1D) and against
  brute-force quadrature of the collision law (2D, 3D) -- arXiv 2506.09465 Sec. 2
  (integral solution, P_f, P_c) and Sec. 3.2 (null collisions reproduce the same law).
* Exact per-sample conservation: net inflow through a cell's faces equals its
  absorbed minus emitted power (Sec. 3.3, Eq. "macro-q-eqn" in integral form).
* Limits: ballistic flux C v dT / 4 between black walls; diffusive slab flux with the
  Milne extrapolation length 0.7104 lambda (Case and Zweifel, Linear Transport Theory).
* The uniform-equilibrium test of Sec. 3.2 (tau jumping by 10^3): T = 1 is preserved.
* Mirror symmetry; W = tau R in expectation (Sec. 3.2, W and W^h).
"""
import numpy as np
import pytest

from oracle import expected as X


def gray_problem(orc, dim, n, L, tau, wall_T, N, Nw=None, seed=0, source=None):
    ncells = int(np.prod(n))
    tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), (ncells,)).reshape(1, -1)
    return orc.Problem(dim, n, L, np.array([1.0]), np.array([1.0]), tau, np.asarray(wall_T, float),
                       np.array([N]), np.array([Nw if Nw is not None else N]), source=source, seed=seed)


def mc_mean(orc, p, T, M, pick):
    acc = np.array([pick(orc.sweep(p, T, e)) for e in range(M)])
    return acc.mean(0), acc.std(0, ddof=1) / np.sqrt(M)


def assert_z(mean, se, exp, zmax=4.5, floor=1e-12):
    z = (mean - exp) / np.maximum(se, floor * np.maximum(1.0, np.abs(exp)))
    assert np.abs(z).max() < zmax, np.round(z, 2)


# ---------------------------------------------------------------------------
# Samplers
# ---------------------------------------------------------------------------

def test_thermal_sampler_moments(orc):
    N = 40000
    p = orc.Problem(3, (3, 2, 2), (1.5, 1.0, 2.0), np.array([1.0]), np.array([2.0]), np.full((1, 12), 0.25),
                    np.zeros(6), np.array([N]), np.array([N]))
    x, s, d = orc.emit(p, 0, 0, 7)  # cell (1, 0, 1)
    h = np.array([0.5, 0.5, 1.0])
    lo = np.array([1, 0, 1]) * h
    frac = (x - lo) / h
    assert np.all((frac > 0) & (frac < 1))
    se = 1.0 / np.sqrt(12 * N)
    assert np.all(np.abs(frac.mean(0) - 0.5) < 5 * se)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    assert np.all(np.abs(s.mean(0)) < 5 / np.sqrt(3 * N))
    assert np.all(np.abs((s ** 2).mean(0) - 1.0 / 3.0) < 5 * np.sqrt(4.0 / 45.0 / N))
    # Path to the first candidate: exponential with mean v tau_maj = 0.5 (Sec. 3.1).
    assert abs(d.mean() - 0.5) < 5 * 0.5 / np.sqrt(N)
    assert abs(np.median(d) - 0.5 * np.log(2.0)) < 0.02
    # Its uniform comes from bits of the emission's Philox block that the position and
    # direction uniforms leave unused: uniform on (0, 1) and uncorrelated with them.
    u = np.exp(-d / 0.5)
    counts, _ = np.histogram(u, bins=32, range=(0.0, 1.0))
    assert ((counts - N / 32) ** 2 / (N / 32)).sum() < 70.0  # 31 dof: p ~ 1e-4
    for v in (frac[:, 0], frac[:, 1], frac[:, 2], s[:, 0]):
        assert abs(np.corrcoef(u, v)[0, 1]) < 5 / np.sqrt(N)


def test_wall_sampler_cosine_law(orc):
    N = 40000
    p = orc.Problem(2, (4, 4), (1.0, 1.0), np.array([1.0]), np.array([1.0]), np.full((1, 16), 0.3),
                    np.zeros(4), np.array([10]), np.array([N]))
    nfx = p.face_counts()[0]
    top = nfx + 1 + 4 * 4  # y-face (ix=1, iy=4): on the +y wall
    x, s, _ = orc.emit(p, 1, 0, top)
    assert np.all(x[:, 1] == 1.0)
    assert np.all((x[:, 0] > 0.25) & (x[:, 0] < 0.5))
    mu_n = -s[:, 1]
    assert np.all(mu_n > 0)
    # Cosine-weighted hemisphere: density 2 mu on (0, 1): E mu = 2/3, E mu^2 = 1/2.
    assert abs(mu_n.mean() - 2.0 / 3.0) < 5 * np.sqrt(1.0 / 18.0 / N)
    assert abs((mu_n ** 2).mean() - 0.5) < 5 * np.sqrt(1.0 / 12.0 / N)
    # 2D keeps the in-plane part of the 3D direction: the z component (sin phi part) is dropped.
    assert np.all(np.linalg.norm(s, axis=1) <= 1.0 + 1e-15)
    # In-plane tangential component s_x = sqrt(1 - mu_n^2) sin(phi): E s_x^2 = (1 - 1/2) / 2.
    assert abs((s[:, 0] ** 2).mean() - 0.25) < 5 * np.sqrt(0.1 / N)


# ---------------------------------------------------------------------------
# 1D: Monte Carlo means against the closed-form E_3 operator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["kn1", "kn01", "jump_null", "two_band"])
def test_slab_sweep_matches_E3(orc, case):
    n, L = 12, 1.0
    T = np.linspace(0.8, -0.3, n)
    wall_T = np.array([1.0, -1.0])
    if case == "kn1":
        C, v, tau, N = [1.0], [1.0], np.ones((1, n)), 300
    elif case == "kn01":
        C, v, tau, N = [1.0], [1.0], np.full((1, n), 0.1), 300
    elif case == "jump_null":  # tau 10 | 0.1 (Sec. 4.2 Case A shape): 100 null candidates per real on the left
        C, v, N = [1.0], [1.0], 200
        tau = np.where(np.arange(n) < n // 2, 10.0, 0.1).reshape(1, n)
    else:  # two bands with different C, v, tau profiles
        C, v, N = [0.6, 1.4], [1.0, 0.5], 200
        tau = np.stack([np.full(n, 0.3), np.linspace(0.05, 0.5, n)])
    p = orc.Problem(1, (n,), (L,), np.array(C), np.array(v), tau, wall_T,
                    np.full(len(C), N), np.full(len(C), N))
    M = 40
    pick = lambda r: np.concatenate([r.R.ravel(), r.W.ravel(), r.F, r.wall])
    mean, se = mc_mean(orc, p, T, M, pick)
    R, W, F, wall = X.slab_expected_sweep(L, C, v, tau, T, wall_T)
    exp = np.concatenate([R.ravel(), W.ravel(), F, wall])
    assert_z(mean, se, exp)


def test_slab_expected_operator_self_consistency():
    # Probabilities of a cell's particle: collide somewhere or escape through a wall.
    t = np.array([0.3, 2.0, 0.05, 1.0, 0.7])
    P, Pw, Xm, Xw = X.slab_probabilities(t)
    esc_right = Xm[-1]              # net crossings of the last face by cell particles
    esc_left = -Xm[0]
    assert np.allclose(P.sum(0) + esc_left + esc_right, 1.0, atol=1e-13)
    # Wall particles: collide or leave through the opposite wall.
    assert np.allclose(Pw[:, 0].sum() + Xw[-1, 0], 1.0, atol=1e-13)
    assert np.allclose(Pw[:, 1].sum() - Xw[0, 1], 1.0, atol=1e-13)
    # Reciprocity of the collision kernel for uniform emission: t_j P_ij = t_i P_ji.
    assert np.allclose(t[None, :] * P, (t[None, :] * P).T, atol=1e-14)


# ---------------------------------------------------------------------------
# 2D / 3D: Monte Carlo means against brute-force quadrature
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_grid2d_sweep_matches_quadrature(orc):
    n, L = (3, 3), (1.0, 1.2)
    tau = np.array([0.5, 0.5, 2.0, 0.2, 0.5, 2.0, 0.2, 0.2, 0.5])
    T = np.array([1.0, 0.2, 0.0, 0.5, 0.0, 0.3, 0.0, 0.7, 0.1])
    wall_T = np.array([0.0, 0.5, 0.2, 1.0])
    Rq = X.grid_expected_R(2, n, L, 1.0, 1.0, tau, T, wall_T, npos=6, nmu=20, nphi=24, nsub=3)
    p = gray_problem(orc, 2, n, L, tau, wall_T, 400)
    mean, se = mc_mean(orc, p, T, 60, lambda r: r.R[0])
    assert_z(mean, se, Rq)


@pytest.mark.slow
def test_grid3d_sweep_matches_quadrature(orc):
    n, L = (2, 2, 2), (1.0, 1.0, 0.8)
    tau = np.array([0.3, 0.3, 1.0, 1.0, 0.3, 0.1, 1.0, 0.3])
    T = np.array([1.0, 0.0, 0.5, 0.0, 0.2, 0.0, 0.0, 0.8])
    wall_T = np.array([0.0, 1.0, 0.0, 0.5, 0.3, 0.0])
    Rq = X.grid_expected_R(3, n, L, 1.0, 1.0, tau, T, wall_T, npos=4, nmu=16, nphi=16, nsub=2)
    p = gray_problem(orc, 3, n, L, tau, wall_T, 300)
    mean, se = mc_mean(orc, p, T, 40, lambda r: r.R[0])
    assert_z(mean, se, Rq)


# ---------------------------------------------------------------------------
# Exact conservation and balance (every sample, rounding only)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_cell_conservation_exact(orc, dim):
    n = {1: (9,), 2: (5, 4), 3: (3, 4, 2)}[dim]
    L = {1: (1.0,), 2: (1.0, 0.7), 3: (1.0, 0.7, 0.5)}[dim]
    rng = np.random.default_rng(dim)
    nc = int(np.prod(n))
    C, v = np.array([0.7, 1.3]), np.array([1.0, 0.6])
    tau = rng.uniform(0.05, 0.8, size=(2, nc))
    wall_T = rng.uniform(-1, 1, size=2 * dim)
    src = rng.uniform(0, 2, size=nc)
    p = orc.Problem(dim, n, L, C, v, tau, wall_T, np.array([40, 60]), np.array([30, 50]), source=src)
    T = rng.uniform(-0.5, 1.0, size=nc)
    r = orc.sweep(p, T, 3)
    V = p.volume()
    m = (C[:, None] / tau).sum(0)
    emitted = (C[:, None] * T[None, :] * V / tau).sum(0) + src * V   # thermal + source (T_emit = T + Q/m)
    # Net inflow from the face tallies.
    nf = p.face_counts()
    off = np.cumsum([0] + nf)
    full = list(n) + [1] * (3 - dim)
    inflow = np.zeros(nc)
    for a in range(dim):
        Fa = r.F[off[a]:off[a + 1]]
        shape = list(full)
        shape[a] += 1
        Fa = Fa.reshape(shape[::-1])  # (z, y, x) with x fastest
        ax = 2 - a
        lo = np.take(Fa, np.arange(full[a]), axis=ax)
        hi = np.take(Fa, np.arange(1, full[a] + 1), axis=ax)
        inflow += (lo - hi).ravel()
    scale = np.abs(r.R).sum() + np.abs(emitted).sum()
    assert np.allclose(inflow, r.R.sum(0) - emitted, atol=1e-12 * scale)
    # Global: absorbed at walls - emitted by walls = emitted in cells - absorbed in cells.
    h = p.h()
    wall_em = 0.0
    for w in range(2 * dim):
        a = w // 2
        area = np.prod([p.L[b] if b < dim else 1.0 for b in range(3) if b != a])
        wall_em += (C * v).sum() * wall_T[w] / 4.0 * area
    assert abs((r.wall.sum() - wall_em) - (emitted.sum() - r.R.sum())) < 1e-12 * scale
    c = r.counters
    assert c[0] == c[2] + c[4] + c[5] and c[5] == 0


def test_W_is_tau_R_in_expectation_and_T_half(orc):
    n = 6
    tau = np.array([[0.2, 1.0, 0.05, 0.4, 0.4, 2.0]])
    p = orc.Problem(1, (n,), (1.0,), np.array([1.0]), np.array([1.0]), tau, np.array([1.0, 0.0]),
                    np.array([400]), np.array([400]))
    T = np.full(n, 0.5)
    mean, se = mc_mean(orc, p, T, 40, lambda r: np.concatenate([r.W[0] - tau[0] * r.R[0]]))
    assert_z(mean, se, np.zeros(n))
    r = orc.sweep(p, T, 0)
    Th, TE = orc.macro(p, r.R, r.W)
    V = 1.0 / n
    assert np.allclose(Th, r.R[0] * tau[0] / V, rtol=1e-14)
    assert np.allclose(TE, r.W[0] / V, rtol=1e-14)


# ---------------------------------------------------------------------------
# Limits and the paper's uniform-equilibrium example
# ---------------------------------------------------------------------------

def test_ballistic_flux_between_black_walls(orc):
    # Kn = 1e6: almost no collisions; every face carries C v (T_H - T_L) / 4.
    n = 20
    p = gray_problem(orc, 1, (n,), (1.0,), 1e6, [1.0, -0.5], 10, Nw=2000)
    r = orc.sweep(p, np.zeros(n), 0)
    assert np.allclose(r.F, (1.0 - (-0.5)) / 4.0, rtol=1e-4)
    # 2D, all walls at 1 except top at 0: interior faces carry no net y-flux on average by symmetry
    # and the expected slab fixed point is (T_H + T_L) / 2 in the ballistic limit.
    T, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], np.full((1, 50), 1e6), [1.0, -0.5])
    assert np.allclose(T, 0.25, atol=1e-4)


def test_diffusive_slab_flux_with_milne_jump():
    # q = k dT / (L + 2 z0 lambda), k = C v lambda / 3, z0 = 0.7104 (Milne problem).
    Kn, n = 0.02, 500
    T, A, b = X.slab_fixed_point(1.0, [1.0], [1.0], np.full((1, n), Kn), [1.0, 0.0])
    _, _, F, _ = X.slab_expected_sweep(1.0, [1.0], [1.0], np.full((1, n), Kn), T, [1.0, 0.0])
    q_ref = (1.0 / 3.0) * Kn * 1.0 / (1.0 + 2 * 0.7104 * Kn)
    assert np.allclose(F, F.mean(), rtol=1e-9)     # div q = 0 at steady state (Sec. 3.3)
    assert abs(F.mean() / q_ref - 1.0) < 0.01
    # Interior profile linear (Fourier), slope -q / k.
    x = (np.arange(n) + 0.5) / n
    mid = slice(n // 5, 4 * n // 5)
    slope = np.polyfit(x[mid], T[mid], 1)[0]
    assert abs(slope / (-F.mean() / (Kn / 3.0)) - 1.0) < 0.01


def test_uniform_equilibrium_preserved_with_tau_jump(orc):
    # Sec. 3.2 example: cells of 0.1, Kn 0.1 left | 1e-4 right, T = 1 everywhere and on both walls.
    n = 10
    tau = np.where(np.arange(n) < 5, 0.1, 1e-4).reshape(1, n)
    T_exp, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], tau, [1.0, 1.0])
    assert np.allclose(T_exp, 1.0, atol=1e-12)
    R, _, F, _ = X.slab_expected_sweep(1.0, [1.0], [1.0], tau, np.ones(n), [1.0, 1.0])
    assert np.allclose(R[0], tau[0] ** -1 * 0.1, rtol=1e-12)   # absorbed = emitted = C T V / tau
    assert np.allclose(F, 0.0, atol=1e-12)
    p = orc.Problem(1, (n,), (1.0,), np.array([1.0]), np.array([1.0]), tau, np.array([1.0, 1.0]),
                    np.array([100]), np.array([100]))
    mean, se = mc_mean(orc, p, np.ones(n), 20, lambda r: orc.macro(p, r.R, r.W)[0])
    assert_z(mean, se, np.ones(n))


def test_mirror_symmetry(orc):
    n = 40
    T, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], np.full((1, n), 0.3), [1.0, -1.0])
    assert np.allclose(T, -T[::-1], atol=1e-12)
    # 2D cavity (top wall hot): MC mean of R is symmetric under x -> 1 - x.
    p = gray_problem(orc, 2, (4, 3), (1.0, 0.75), 0.3, [0.0, 0.0, 0.0, 1.0], 200)
    mean, se = mc_mean(orc, p, np.zeros(12), 40, lambda r: r.R[0].reshape(3, 4))
    d = mean - mean[:, ::-1]
    assert np.all(np.abs(d) < 5 * np.sqrt(2) * se + 1e-15)


def test_band_split(orc):
    r = np.array([1.0, 10.0, 0.01, 3.0])
    s = orc.band_split(1000, r)
    assert s.sum() == 1000 and np.all(s >= 1)
    ideal = 1 + (1000 - 4) * r / r.sum()
    assert np.all(np.abs(s - ideal) <= 1.0)
    with pytest.raises(ValueError):
        orc.band_split(3, r)


# ---------------------------------------------------------------------------
# Per-face wall temperatures (the non-uniform boundary of Sec. 4.5)
# ---------------------------------------------------------------------------

def _rect(orc, n=(20, 10), L=(5.0, 2.5), tau=1e9, N=64, face_T=None, wall_T=(0.0, 0.0, 0.0, 0.0), seed=3):
    nc = n[0] * n[1]
    return orc.Problem(2, n, L, np.array([1.0]), np.array([1.0]), np.full((1, nc), tau), np.array(wall_T),
                       np.array([N]), np.array([N]), seed=seed, wall_face_T=face_T)


def test_face_temperatures_equal_to_wall_values_reproduce_wall_sweep(orc):
    wall_T = np.array([0.3, -0.2, 0.1, 1.0])
    base = _rect(orc, tau=0.7, wall_T=wall_T)
    faces = np.concatenate([np.full(m, t) for m, t in zip(base.wall_faces(), wall_T)])
    per_face = _rect(orc, tau=0.7, wall_T=wall_T, face_T=faces)
    T = np.linspace(0, 1, 200)
    a, b = orc.sweep(base, T, 0), orc.sweep(per_face, T, 0)
    for x, y in ((a.R, b.R), (a.W, b.W), (a.F, b.F), (a.wall, b.wall)):
        assert np.array_equal(x, y)


def test_face_temperatures_superpose(orc):
    # The sweep is linear in the emission and draws are keyed by (emitter, particle): the
    # sum over the top wall's faces of one-hot-face sweeps is the uniform-wall sweep.
    n, L = (6, 4), (1.5, 1.0)
    base = _rect(orc, n=n, L=L, tau=0.4, wall_T=(0.0, 0.0, 0.0, 1.0))
    nf = base.wall_faces()
    off = sum(nf[:3])
    acc = None
    for j in range(nf[3]):
        ft = np.zeros(sum(nf))
        ft[off + j] = 1.0
        r = orc.sweep(_rect(orc, n=n, L=L, tau=0.4, face_T=ft), np.zeros(24), 0)
        v = np.concatenate([r.R.ravel(), r.W.ravel(), r.F, r.wall])
        acc = v if acc is None else acc + v
    r = orc.sweep(base, np.zeros(24), 0)
    ref = np.concatenate([r.R.ravel(), r.W.ravel(), r.F, r.wall])
    assert np.allclose(acc, ref, rtol=1e-12, atol=1e-15)


def test_hot_segment_ballistic_view_factors(orc):
    # Sec. 4.5 geometry, L_x = 2 L_y = 5 L_1: a hot segment of length L_1 centred on the top
    # wall, no collisions (tau = 1e9). The power it emits is absorbed by the other walls in
    # the proportions of the 2D (crossed-strings) view factors of a diffuse emitter.
    Lx, Ly = 5.0, 2.5
    n = (20, 10)
    ft = np.zeros(2 * n[1] + 2 * n[0])
    top = 2 * n[1] + n[0]
    ft[top + 8: top + 12] = 1.0                      # x in [2, 3]
    N = 4000
    r = orc.sweep(_rect(orc, n=n, L=(Lx, Ly), N=N, face_T=ft), np.zeros(200), 0)
    emitted = 1.0 * 1.0 * 1.0 / 4.0                  # C v T L_1 / 4 per unit depth
    assert abs(r.wall.sum() - emitted) < 1e-12
    d = lambda p, q: np.hypot(p[0] - q[0], p[1] - q[1])

    def view(a1, a2, b1, b2):  # crossed strings, segment a1-a2 to b1-b2, per unit length of a
        return (d(a1, b2) + d(a2, b1) - d(a1, b1) - d(a2, b2)) / (2.0 * d(a1, a2))

    a1, a2 = (2.0, Ly), (3.0, Ly)
    F = {0: abs(view(a1, a2, (0.0, Ly), (0.0, 0.0))),    # left wall
         1: abs(view(a1, a2, (Lx, 0.0), (Lx, Ly))),      # right wall
         2: abs(view(a1, a2, (0.0, 0.0), (Lx, 0.0)))}    # bottom wall
    assert abs(sum(F.values()) - 1.0) < 1e-12
    for wall, f in F.items():
        frac = r.wall[wall] / emitted
        se = np.sqrt(f * (1 - f) / (4 * N))
        assert abs(frac - f) < 4.5 * se, (wall, frac, f)
    assert r.wall[3] == 0.0
