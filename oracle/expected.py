"""Expected (infinite-particle) operator of one IUGKP sweep, computed without Monte Carlo.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``). Used to pin the Monte Carlo oracle:
the mean of the oracle's sweep tallies over many independent epochs must agree with
these deterministic values within its standard error.

The sweep is the particle form of the integral solution of the steady BGK equation
(arXiv 2506.09465, Sec. 2, integral solution and Eqs. "sum-g" / "sum-g-CDF"): a
particle emitted at x0 in direction s has its real collision between path lengths r
and r + dr with density sigma(r) exp(-int_0^r sigma), sigma = 1 / (v tau(x))
(Sec. 2, P_f and P_c; Sec. 3.2 shows that null collisions reproduce the same law,
Eq. for f(s)). With tau piecewise constant per cell the probability of the real
collision falling in the k-th cell crossed is exp(-tau_in) - exp(-tau_out), tau_in /
tau_out being the optical depths at entry and exit.

* 1D (slab): integrating that law over a uniform emission position and mu ~ U(-1, 1)
  gives closed forms in the exponential integral E_3 (E_n(x) = int_1^inf e^{-xt} t^-n dt,
  with d/dx E_3 = -E_2 and int_0^1 e^{-a/mu} mu^{n-2} dmu = E_n(a)).
* 2D / 3D (tiny grids): brute-force tensor Gauss-Legendre quadrature over the emission
  position and the direction, each ray walked cell by cell exactly.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expn


def E3(x):
    return expn(3, np.asarray(x, dtype=np.float64))


# ---------------------------------------------------------------------------
# 1D slab: collision probabilities in closed form
# ---------------------------------------------------------------------------

def slab_probabilities(t: np.ndarray):
    """t[k]: optical thickness of cell k (h / (v tau_k)).

    Returns (P, Pw, X, Xw):
      P[i, j]  = probability that a particle emitted uniformly in cell j, mu ~ U(-1,1),
                 has its real collision in cell i;
      Pw[i, w] = same for a particle from wall w (0 = left at x=0, 1 = right),
                 cosine-weighted (mu density 2 mu on (0, 1));
      X[k, j]  = expected net crossings of face k (+x minus -x) by a particle of cell j;
      Xw[k, w] = same for wall w.
    """
    n = len(t)
    edges = np.concatenate([[0.0], np.cumsum(t)])  # optical coordinate of faces 0..n
    P = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            if i == j:
                P[i, j] = 1.0 - (0.5 - E3(t[j])) / t[j]
            else:
                if i > j:
                    g = edges[i] - edges[j + 1]
                else:
                    g = edges[j] - edges[i + 1]
                P[i, j] = (E3(g) - E3(g + t[i]) - E3(g + t[j]) + E3(g + t[i] + t[j])) / (2.0 * t[j])
    Pw = np.zeros((n, 2))
    for i in range(n):
        gl = edges[i]
        gr = edges[n] - edges[i + 1]
        Pw[i, 0] = 2.0 * (E3(gl) - E3(gl + t[i]))
        Pw[i, 1] = 2.0 * (E3(gr) - E3(gr + t[i]))
    X = np.zeros((n + 1, n))
    for j in range(n):
        for k in range(n + 1):
            if k >= j + 1:  # face to the right of cell j: crossed by right-movers
                g = edges[k] - edges[j + 1]
                X[k, j] = (E3(g) - E3(g + t[j])) / (2.0 * t[j])
            elif k <= j:  # face to the left: crossed by left-movers (negative)
                g = edges[j] - edges[k]
                X[k, j] = -(E3(g) - E3(g + t[j])) / (2.0 * t[j])
    Xw = np.zeros((n + 1, 2))
    for k in range(n + 1):
        Xw[k, 0] = 2.0 * E3(edges[k])               # from the left wall, moving +x
        Xw[k, 1] = -2.0 * E3(edges[n] - edges[k])    # from the right wall, moving -x
    return P, Pw, X, Xw


def slab_expected_sweep(L: float, C, v, tau, T_emit, wall_T):
    """Expected tallies of one 1D sweep: R [nb, n], W [nb, n], F [n+1], wall [2].

    Emission powers (per unit area): cell C_b T V / tau_b, wall C_b v_b T_w / 4.
    """
    C = np.atleast_1d(np.asarray(C, dtype=np.float64))
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    tau = np.asarray(tau, dtype=np.float64).reshape(len(C), -1)
    nb, n = tau.shape
    h = L / n
    R = np.zeros((nb, n))
    W = np.zeros((nb, n))
    F = np.zeros(n + 1)
    wall = np.zeros(2)
    for b in range(nb):
        t = h / (v[b] * tau[b])
        P, Pw, X, Xw = slab_probabilities(t)
        S = C[b] * np.asarray(T_emit) * h / tau[b]
        Sw = C[b] * v[b] * np.asarray(wall_T) / 4.0
        R[b] = P @ S + Pw @ Sw
        W[b] = tau[b] * R[b]   # candidates per unit track are 1/(v tau_maj), real ones 1/(v tau)
        Fb = X @ S + Xw @ Sw
        F += Fb
        # Absorbed by a wall = power leaving through its end face: the net crossing of
        # that face plus the wall's own emission, which crosses it inwards.
        wall[0] += Sw[0] - Fb[0]
        wall[1] += Fb[n] + Sw[1]
    return R, W, F, wall


def slab_fixed_point(L: float, C, v, tau, wall_T, source=None):
    """Steady state of the expected iteration T = A T + b in 1D (dense solve).

    T_half[i] = sum_b R_b[i] / (V m_i) with m_i = sum_b C_b / tau_{b,i}.
    """
    C = np.atleast_1d(np.asarray(C, dtype=np.float64))
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    tau = np.asarray(tau, dtype=np.float64).reshape(len(C), -1)
    nb, n = tau.shape
    h = L / n
    m = (C[:, None] / tau).sum(axis=0)
    A = np.zeros((n, n))
    b = np.zeros(n)
    for k in range(nb):
        t = h / (v[k] * tau[k])
        P, Pw, _, _ = slab_probabilities(t)
        coef = C[k] * h / tau[k]                     # emitted power per unit T_emit
        A += P * coef[None, :]
        b += Pw @ (C[k] * v[k] * np.asarray(wall_T) / 4.0)
    A /= (h * m)[:, None]
    b /= h * m
    if source is not None:
        b += A @ (np.asarray(source) / m)   # the source shifts the emission temperature by Q/m
    T = np.linalg.solve(np.eye(n) - A, b)
    return T, A, b


# ---------------------------------------------------------------------------
# 2D / 3D: brute-force quadrature of the same collision law
# ---------------------------------------------------------------------------

def _gl(npts, a, b):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _walk(dim, n, h, sig, x0, s, ncell_idx):
    """Exact walk of rays (vectorised). x0: [R, 3] start points, s: [R, 3] directions,
    ncell_idx: [R, 3] int start cells. sig: [ncells] (1 / (v tau)) per cell.
    Returns prob [R, ncells]: probability of the real collision in each cell."""
    nr = x0.shape[0]
    nc = sig.size
    prob = np.zeros((nr, nc))
    x = x0.copy()
    idx = ncell_idx.copy()
    depth = np.zeros(nr)
    alive = np.ones(nr, dtype=bool)
    steps = 0
    while alive.any():
        steps += 1
        assert steps < 10 * sum(n) + 10
        tmin = np.full(nr, np.inf)
        amin = np.zeros(nr, dtype=np.int64)
        for a in range(dim):
            with np.errstate(divide="ignore", invalid="ignore"):
                up = ((idx[:, a] + 1) * h[a] - x[:, a]) / s[:, a]
                dn = (idx[:, a] * h[a] - x[:, a]) / s[:, a]
            ta = np.where(s[:, a] > 0, up, np.where(s[:, a] < 0, dn, np.inf))
            better = ta < tmin
            tmin = np.where(better, ta, tmin)
            amin = np.where(better, a, amin)
        c = idx[:, 0] + n[0] * (idx[:, 1] + n[1] * idx[:, 2])
        ci = np.where(alive, c, 0)
        d_out = depth + tmin * sig[ci]
        p = np.exp(-depth) - np.exp(-d_out)
        rows = np.nonzero(alive)[0]
        np.add.at(prob, (rows, ci[rows]), p[rows])
        depth = d_out
        x = x + tmin[:, None] * s
        step = np.where(s[np.arange(nr), amin] > 0, 1, -1)
        idx[np.arange(nr), amin] += step
        out = (idx[np.arange(nr), amin] < 0) | (idx[np.arange(nr), amin] >= np.asarray(n)[amin])
        alive &= ~out
        idx = np.where(alive[:, None], idx, 0)
        x = np.where(alive[:, None], x, 0.5 * np.asarray(h)[None, :])
    return prob


def quadrature_operator(dim, n, L, tau, v, npos=6, nmu=24, nphi=24, nsub=2):
    """Collision probabilities by quadrature for a gray medium on a tiny 2D/3D grid.

    Returns (K, Kw): K[i, j] for cell emitters (uniform position, isotropic direction),
    Kw[i, f] for wall emitters, one column per wall (-x, +x, -y, +y, -z, +z): a wall's
    column averages over its faces weighted by area (cosine-weighted directions).
    Each emitting cell is split into nsub^dim sub-cells with npos Gauss points per axis;
    mu uses nmu Gauss points on each of (-1, 0) and (0, 1) and phi nphi points.
    """
    n = list(n) + [1] * (3 - len(n))
    L = list(L) + [1.0] * (3 - len(L))
    h = [L[a] / n[a] if a < dim else 1.0 for a in range(3)]
    ncells = n[0] * n[1] * n[2]
    sig = 1.0 / (v * np.asarray(tau, dtype=np.float64).reshape(-1))
    # Direction quadrature (3D isotropic; density 1/(4 pi) in mu, phi).
    mu_a, wmu_a = _gl(nmu, -1.0, 0.0)
    mu_b, wmu_b = _gl(nmu, 0.0, 1.0)
    mu = np.concatenate([mu_a, mu_b])
    wmu = np.concatenate([wmu_a, wmu_b]) / 2.0
    phi, wphi = _gl(nphi, 0.0, 2.0 * np.pi)
    wphi = wphi / (2.0 * np.pi)
    if dim == 1:
        phi, wphi = np.array([0.0]), np.array([1.0])
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    WD = np.outer(wmu, wphi).ravel()
    sn = np.sqrt(1.0 - MU.ravel() ** 2)
    S = np.stack([MU.ravel(), sn * np.cos(PHI.ravel()), sn * np.sin(PHI.ravel())], axis=1)
    if dim < 3:
        S[:, 2] = 0.0
    if dim < 2:
        S[:, 1] = 0.0
    # Position quadrature inside a unit cell.
    gp, gw = _gl(npos, 0.0, 1.0)
    sub_x = np.concatenate([(k + gp) / nsub for k in range(nsub)])
    sub_w = np.concatenate([gw / nsub for _ in range(nsub)])
    axes_pts = [sub_x if a < dim else np.array([0.5]) for a in range(3)]
    axes_w = [sub_w if a < dim else np.array([1.0]) for a in range(3)]
    PX, PY, PZ = np.meshgrid(*axes_pts, indexing="ij")
    WP = np.einsum("i,j,k->ijk", *axes_w).ravel()
    frac = np.stack([PX.ravel(), PY.ravel(), PZ.ravel()], axis=1)
    K = np.zeros((ncells, ncells))
    for j in range(ncells):
        cj = np.array([j % n[0], (j // n[0]) % n[1], j // (n[0] * n[1])])
        x0 = (cj[None, :] + frac) * np.asarray(h)[None, :]
        X0 = np.repeat(x0, S.shape[0], axis=0)
        SS = np.tile(S, (x0.shape[0], 1))
        W8 = np.outer(WP, WD).ravel()
        IDX = np.repeat(np.tile(cj, (x0.shape[0], 1)), S.shape[0], axis=0)
        prob = _walk(dim, n, h, sig, X0, SS, IDX)
        K[:, j] = (prob * W8[:, None]).sum(axis=0)
    # Wall emitters: cosine-weighted into the domain.
    nw = 2 * dim
    Kw = np.zeros((ncells, nw))
    un, wun = _gl(nmu, 0.0, 1.0)        # u_n uniform; mu_n = sqrt(u_n) is cosine-weighted
    for wall in range(nw):
        a, side = wall // 2, wall % 2
        o1, o2 = (a + 1) % 3, (a + 2) % 3
        dirs = []
        wts = []
        for iu, u in enumerate(un):
            for ip, ph in enumerate(phi):
                s = np.zeros(3)
                s[a] = np.sqrt(u) if side == 0 else -np.sqrt(u)
                st = np.sqrt(1.0 - u)
                s[o1] = st * np.cos(ph)
                s[o2] = st * np.sin(ph)
                for ax in range(dim, 3):
                    s[ax] = 0.0
                dirs.append(s)
                wts.append(wun[iu] * wphi[ip])
        dirs = np.array(dirs)
        wts = np.array(wts)
        # Faces of this wall; positions along the tangential in-domain axes.
        tang = [ax for ax in sorted((o1, o2)) if ax < dim]
        face_cells = []
        for j2 in range(n[o2]):
            for j1 in range(n[o1]):
                f = [0, 0, 0]
                f[a] = 0 if side == 0 else n[a] - 1
                f[o1], f[o2] = j1, j2
                face_cells.append(f)
        nf = len(face_cells)
        tp = [sub_x if ax in tang else np.array([0.5]) for ax in (o1, o2)]
        tw = [sub_w if ax in tang else np.array([1.0]) for ax in (o1, o2)]
        T1, T2 = np.meshgrid(tp[0], tp[1], indexing="ij")
        TW = np.outer(tw[0], tw[1]).ravel()
        for f in face_cells:
            x0 = np.zeros((T1.size, 3))
            x0[:, a] = 0.0 if side == 0 else L[a]
            x0[:, o1] = (f[o1] + T1.ravel()) * h[o1]
            x0[:, o2] = (f[o2] + T2.ravel()) * h[o2]
            for ax in range(dim, 3):
                x0[:, ax] = 0.5
            X0 = np.repeat(x0, dirs.shape[0], axis=0)
            SS = np.tile(dirs, (x0.shape[0], 1))
            W8 = np.outer(TW, wts).ravel()
            IDX = np.repeat(np.tile(np.array(f), (x0.shape[0], 1)), dirs.shape[0], axis=0)
            prob = _walk(dim, n, h, sig, X0, SS, IDX)
            Kw[:, wall] += (prob * W8[:, None]).sum(axis=0) / nf
    return K, Kw


def grid_expected_R(dim, n, L, C, v, tau, T_emit, wall_T, **quad):
    """Expected R per cell (gray) from the quadrature operator."""
    n3 = list(n) + [1] * (3 - len(n))
    L3 = list(L) + [1.0] * (3 - len(L))
    h = [L3[a] / n3[a] if a < dim else 1.0 for a in range(3)]
    V = h[0] * h[1] * h[2]
    tau = np.asarray(tau, dtype=np.float64).reshape(-1)
    K, Kw = quadrature_operator(dim, n, L, tau, v, **quad)
    S = C * np.asarray(T_emit) * V / tau
    # Power of one wall: C v T_w / 4 times its total area.
    area = []
    for wall in range(2 * dim):
        a = wall // 2
        tot = 1.0
        for ax in range(3):
            if ax != a:
                tot *= L3[ax] if ax < dim else 1.0
        area.append(tot)
    Sw = C * v * np.asarray(wall_T) / 4.0 * np.asarray(area)
    return K @ S + Kw @ Sw
