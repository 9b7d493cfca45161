"""Checks against stored values: the paper's printed tables and the expected steady
state of the 1D slab written by tests/golden/make_golden.py (oracle only)."""
import os

import numpy as np
import pytest

from oracle import expected as X

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_paper_speedups_follow_the_stated_formula():
    # R_s = N_wp / N_current * R_e with R_e = 4 reproduces every printed speedup to the
    # paper's rounding (Sec. 4, speedup formula; Tables 1-6).
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_tables.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 19
    for _, _, nwp, ncur, printed in rows:
        rs = float(nwp) / float(ncur) * 4.0
        assert abs(rs - float(printed)) <= 0.02 * float(printed) + 1.0, (nwp, ncur, printed, rs)


def load_slab():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "slab_kn1_50cells.txt")) if l[0] != "#"]
    return np.array([float(r[1]) for r in rows])


def test_golden_slab_matches_expected_module():
    T = load_slab()
    T2, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], np.ones((1, 50)), [1.0, -1.0])
    assert np.allclose(T, T2, rtol=1e-13, atol=1e-14)
    assert np.allclose(T, -T[::-1], atol=1e-12)
    assert 0.0 < T[0] < 1.0 and np.all(np.diff(T) < 0)


@pytest.mark.slow
def test_oracle_frozen_fixed_points_average_to_golden(orc):
    # Each seed gives the fixed point of its own frozen-draw map; their mean converges to
    # the expected steady state (Sec. 4.1 setup, 1000 particles per cell).
    T_gold = load_slab()
    n, M = 50, 12
    sols = []
    for seed in range(M):
        p = orc.Problem(1, (n,), (1.0,), np.array([1.0]), np.array([1.0]), np.ones((1, n)), np.array([1.0, -1.0]),
                        np.array([1000]), np.array([1000]), seed=seed)
        T, it, res, _ = orc.solve_steady(p, np.zeros(n), 1e-8, 100, frozen=True, newton=False, dT_ref=2.0)
        assert res <= 1e-8 and it < 40
        sols.append(T)
    sols = np.array(sols)
    z = (sols.mean(0) - T_gold) / (sols.std(0, ddof=1) / np.sqrt(M))
    assert np.abs(z).max() < 4.5


def load_variable_tau(name):
    path = os.path.join(GOLDEN, name)
    rows = np.array([[float(v) for v in l.split()] for l in open(path) if l[0] != "#"])
    q = float([l for l in open(path) if "heat flux" in l][0].split(":")[1])
    return rows[:, 0], rows[:, 1], rows[:, 2], q


@pytest.mark.parametrize("name", ["slab_jump_caseA_100cells.txt", "slab_jump_caseB_100cells.txt",
                                  "slab_multiscale_100cells.txt"])
def test_variable_tau_golden_profiles(name):
    # Stored steady states of the variable-tau films (Sec. 4.2, 4.3) equal the expected-
    # operator fixed point, and at that state the net flux is the same through every face
    # (zero divergence: what a steady state means).
    x, tau, T, q = load_variable_tau(name)
    xc = (np.arange(100) + 0.5) / 100
    if "multiscale" in name:
        tau_def = 10.0 ** (np.abs(2.0 * np.sin(2.0 * np.pi * xc)) - 1.0)
    else:
        tau_def = np.where(xc < 0.5, 10.0, 0.1 if "caseA" in name else 1.0)
    assert np.allclose(tau, tau_def, rtol=1e-14)
    T2, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], tau_def.reshape(1, -1), [1.0, -1.0])
    assert np.allclose(T, T2, rtol=1e-13, atol=1e-14)
    _, _, F, wall = X.slab_expected_sweep(1.0, [1.0], [1.0], tau.reshape(1, -1), T, [1.0, -1.0])
    assert np.abs(F - q).max() <= 1e-10 * abs(q)
    assert abs(wall.sum()) <= 1e-10 * abs(q)   # what one wall emits net, the other absorbs
    assert np.all(np.diff(T) < 0) and 0 < q < 0.5   # below the ballistic limit C v dT / 4


def test_multiscale_profile_is_antisymmetric():
    # tau(x) = 10^(|2 sin 2 pi x| - 1) is symmetric about x = 1/2 and the walls are +-1.
    _, tau, T, _ = load_variable_tau("slab_multiscale_100cells.txt")
    assert np.allclose(tau, tau[::-1], rtol=1e-12)
    assert np.abs(T + T[::-1]).max() < 1e-11


def test_case_A_thick_half_follows_fourier():
    # In the tau = 0.1 half (Kn 0.1), 1.5 mean free paths from the interface and the wall,
    # the profile is linear with the slope of Fourier's law, k = C v^2 tau / 3.
    x, tau, T, q = load_variable_tau("slab_jump_caseA_100cells.txt")
    sel = (x > 0.65) & (x < 0.85)
    slope = np.polyfit(x[sel], T[sel], 1)[0]
    assert abs(slope / (-q / (0.1 / 3.0)) - 1.0) < 0.01


def test_oracle_statistical_average_matches_expected_steady_state(orc):
    # Averaging after convergence (Sec. 4.4): with fresh draws each iteration is a random
    # affine map whose expectation has the stored steady state as fixed point, so the mean
    # of the iterates converges to it. Standard error from 20 batch means of 20 steps
    # (successive iterates are correlated); the face flux averages to the stored flux.
    T_gold = load_slab()
    q_gold = float([l for l in open(os.path.join(GOLDEN, "slab_kn1_50cells.txt")) if "heat flux" in l][0]
                   .split(":")[1])
    n = 50
    p = orc.Problem(1, (n,), (1.0,), np.array([1.0]), np.array([1.0]), np.ones((1, n)), np.array([1.0, -1.0]),
                    np.array([200]), np.array([200]), seed=4)
    T0, _, _, _ = orc.solve_steady(p, np.zeros(n), 1e-8, 200, frozen=True, newton=True, dT_ref=2.0)
    nb, bl = 20, 20
    means, fluxes = [], []
    T = T0
    for b in range(nb):
        T, Tm, Tv, Fm = orc.average(p, T, bl, 1000 + b * bl)
        means.append(Tm)
        fluxes.append(Fm.mean())
        assert np.all(Tv > 0)
    means = np.array(means)
    z = (means.mean(0) - T_gold) / (means.std(0, ddof=1) / np.sqrt(nb))
    assert np.abs(z).max() < 4.5
    fluxes = np.array(fluxes)
    assert abs(fluxes.mean() - q_gold) < 4.5 * fluxes.std(ddof=1) / np.sqrt(nb)
    # one call over all the steps = the pooled batches (same draws, same order)
    _, Tm_all, _, _ = orc.average(p, T0, nb * bl, 1000)
    assert np.allclose(Tm_all, means.mean(0), rtol=1e-12, atol=1e-14)
