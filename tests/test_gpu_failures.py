"""Failure detection on the GPU without a device fault: limits that end work early are
reported through status codes read on the host, and the context stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_09465_gb300 import workloads as WL  # noqa: E402
from gpu_helpers import gpu_solver  # noqa: E402


def test_step_budget_drops_particles_and_reports():
    from paper_2506_09465_gb300._lib import IugkpError
    inst = WL.cavity(16, 1.0).instances[0]
    s = gpu_solver(inst, [1.0], [1.0], 32, 32, precision=0, tally=0, schedule=0, step_budget=3)
    T = torch.full((inst.ncells,), 0.5, dtype=torch.float64, device="cuda")
    with pytest.raises(IugkpError) as e:
        s.sweep(T, 0)
    assert e.value.status == 5 and "budget" in str(e.value)
    # the device error word was reset: a context with a normal budget still works
    s2 = gpu_solver(inst, [1.0], [1.0], 32, 32, precision=0, tally=0, schedule=0)
    g = s2.sweep(T, 0)
    assert g["counters"].cpu().numpy()[5] == 0


def test_cg_cap_reported_as_no_convergence():
    from paper_2506_09465_gb300._lib import IugkpError
    inst = WL.cavity(32, 0.1).instances[0]
    s = gpu_solver(inst, [1.0], [1.0], 32, 32, cg_rtol=1e-14, cg_maxit=1)
    T = torch.full((inst.ncells,), 0.5, dtype=torch.float64, device="cuda")
    g = s.sweep(T, 0)
    Th, _ = s.macro(g["R"])
    with pytest.raises(IugkpError) as e:
        s.newton_step(T, Th, g["R"])
    assert e.value.status == 4
    with pytest.raises(IugkpError) as e:
        s.solve_steady(None, 1e-8, 4)
    assert e.value.status == 4
    g2 = s.sweep(T, 0)  # still usable
    assert g2["counters"].cpu().numpy()[0] > 0


def test_max_iter_reported():
    inst = WL.cavity(16, 1.0).instances[0]
    s = gpu_solver(inst, [1.0], [1.0], 32, 32)
    T, it, res = s.solve_steady(None, 1e-30, 4, raise_on_noconv=False)
    assert it == 4 and res > 1e-30
