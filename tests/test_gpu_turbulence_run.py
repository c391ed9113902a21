"""The driven-turbulence run driver (paper_1602_09079_gb300.turbulence) on
a small box: driving from rest raises the rms Mach number, and the energy
budget closes (total energy change = injected work - dissipated energy)."""
import pytest

pytestmark = pytest.mark.gpu


def test_short_driven_run_energy_budget():
    import torch
    assert torch.cuda.is_available()
    from paper_1602_09079_gb300 import turbulence
    res = turbulence.run(n=16, order=3, gamma=1.01, t_end=0.3, record_every=0.1)
    s = res["summary"]
    assert res["steps"] > 10
    assert 0.0 < s["rms_mach_final"] < 1.0
    assert s["injected"] > 0.0
    assert abs(s["budget_residual"]) <= 1e-3 * (abs(s["injected"]) + abs(s["dissipated"]))
