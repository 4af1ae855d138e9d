"""Host logic of the Taylor-Green driver (no GPU): the CFL time step of
Sec. 2 and Sec. 4.1, dt = Cr / k_u^1.5 * h / U0."""
import math

import pytest


def test_cfl_time_step_formula():
    from paper_1802_01439_gb300.tgv import cfl_time_step
    assert cfl_time_step(3, 2 * math.pi / 8) == pytest.approx(0.125 / 3 ** 1.5 * 2 * math.pi / 8, rel=1e-15)
    # halving h or doubling |u|_max halves the step; Cr scales it linearly
    assert cfl_time_step(4, 0.1, u_max=2.0) == pytest.approx(0.5 * cfl_time_step(4, 0.1), rel=1e-15)
    assert cfl_time_step(4, 0.05) == pytest.approx(0.5 * cfl_time_step(4, 0.1), rel=1e-15)
    assert cfl_time_step(2, 0.1, courant=0.25) == pytest.approx(2 * cfl_time_step(2, 0.1), rel=1e-15)
