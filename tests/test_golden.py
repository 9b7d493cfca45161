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
