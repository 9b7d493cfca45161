"""Writes the stored expected values under tests/golden/.

Calls only oracle/ (the deterministic expected-operator module); never the CUDA path.
Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import expected as X  # noqa: E402


def slab_config():
    # Gray slab of Sec. 4.1 shape: L = 1, C = |v| = 1, tau = 1 (Kn = 1), 50 cells,
    # black walls at deviational T = +1 (x = 0) and -1 (x = 1).
    n = 50
    T, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], np.ones((1, n)), [1.0, -1.0])
    _, _, F, _ = X.slab_expected_sweep(1.0, [1.0], [1.0], np.ones((1, n)), T, [1.0, -1.0])
    path = os.path.join(HERE, "slab_kn1_50cells.txt")
    with open(path, "w") as f:
        f.write("# Expected (infinite-particle) steady state of the 1D gray slab: 50 cells on [0,1],\n")
        f.write("# C = v = 1, tau = 1 (Kn = 1), walls T = +1 / -1. Written by tests/golden/make_golden.py\n")
        f.write("# from the E_3 closed-form operator (oracle/expected.py); method: arXiv 2506.09465 Sec. 2-3.1.\n")
        f.write(f"# heat flux (constant across faces at steady state): {F.mean():.15e}\n")
        f.write("# cell_centre T\n")
        for i in range(n):
            f.write(f"{(i + 0.5) / n:.6f} {T[i]:.15e}\n")


def variable_tau_configs():
    # The variable-tau films of Sec. 4.2 (tau 10 | 0.1 and 10 | 1, "Case A" and "Case B")
    # and Sec. 4.3 (tau = 10^(|2 sin(2 pi x)| - 1)): 100 cells on [0, 1], C = v = 1, walls
    # T = +1 / -1; tau evaluated at the cell centres.
    n = 100
    x = (np.arange(n) + 0.5) / n
    cases = {
        "slab_jump_caseA_100cells.txt": ("tau = 10 for x < 1/2, 0.1 for x > 1/2 (Sec. 4.2 Case A)",
                                         np.where(x < 0.5, 10.0, 0.1)),
        "slab_jump_caseB_100cells.txt": ("tau = 10 for x < 1/2, 1 for x > 1/2 (Sec. 4.2 Case B)",
                                         np.where(x < 0.5, 10.0, 1.0)),
        "slab_multiscale_100cells.txt": ("tau = 10^(|2 sin(2 pi x)| - 1) at cell centres (Sec. 4.3)",
                                         10.0 ** (np.abs(2.0 * np.sin(2.0 * np.pi * x)) - 1.0)),
    }
    for name, (what, tau) in cases.items():
        tau = tau.reshape(1, n)
        T, _, _ = X.slab_fixed_point(1.0, [1.0], [1.0], tau, [1.0, -1.0])
        _, _, F, _ = X.slab_expected_sweep(1.0, [1.0], [1.0], tau, T, [1.0, -1.0])
        with open(os.path.join(HERE, name), "w") as f:
            f.write("# Expected (infinite-particle) steady state of a 1D gray slab: 100 cells on [0,1],\n")
            f.write(f"# C = v = 1, {what}, walls T = +1 / -1.\n")
            f.write("# Written by tests/golden/make_golden.py from the E_3 closed-form operator\n")
            f.write("# (oracle/expected.py); method: arXiv 2506.09465 Sec. 2-3.2.\n")
            f.write(f"# heat flux (constant across faces at steady state): {F.mean():.15e}\n")
            f.write("# cell_centre tau T\n")
            for i in range(n):
                f.write(f"{x[i]:.6f} {tau[0, i]:.15e} {T[i]:.15e}\n")


if __name__ == "__main__":
    slab_config()
    variable_tau_configs()
