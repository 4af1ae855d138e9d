"""Host logic of the drivers (no GPU): the CFL time step of the
Taylor-Green driver (Sec. 2 and Sec. 4.1, dt = Cr / k_u^1.5 * h / U0), its
kinetic-energy normalisation, and the mesh sizes of the degree sweep."""
import math

import pytest


def test_cfl_time_step_formula():
    from paper_1802_01439_gb300.tgv import cfl_time_step
    assert cfl_time_step(3, 2 * math.pi / 8) == pytest.approx(0.125 / 3 ** 1.5 * 2 * math.pi / 8, rel=1e-15)
    # halving h or doubling |u|_max halves the step; Cr scales it linearly
    assert cfl_time_step(4, 0.1, u_max=2.0) == pytest.approx(0.5 * cfl_time_step(4, 0.1), rel=1e-15)
    assert cfl_time_step(4, 0.05) == pytest.approx(0.5 * cfl_time_step(4, 0.1), rel=1e-15)
    assert cfl_time_step(2, 0.1, courant=0.25) == pytest.approx(2 * cfl_time_step(2, 0.1), rel=1e-15)


def test_degree_sweep_sizes():
    """The degree sweep's meshes: n = round(256 / (k+1)) cells per direction,
    so every k = 2..11 has n^3 (k+1)^3 within 5 % of 2^24 (16.8M) scalar DoFs
    (k = 3 on 64^3 cells, k = 7 on 32^3 exactly)."""
    from paper_1802_01439_gb300.opbench import SWEEP_N
    assert sorted(SWEEP_N) == list(range(2, 12))
    for k, n in SWEEP_N.items():
        assert n == round(256 / (k + 1))
        assert abs(n ** 3 * (k + 1) ** 3 / 2 ** 24 - 1) <= 0.05, (k, n)
    assert SWEEP_N[3] == 64 and SWEEP_N[7] == 32


def test_kinetic_energy_normalisation():
    """tgv.kinetic_energy = u^T M u / (2 |Omega|) on the [-pi, pi]^3 box, the
    oracle's e_k (Sec. 4), computed through the oracle-backed test double of
    the library's mass matrix and dot product."""
    import numpy as np
    import torch
    from oracle import dg
    from paper_1802_01439_gb300.tgv import kinetic_energy
    from tests.host_double import OracleContext
    m = dg.Mesh(2)
    ctx = OracleContext(m, 3, 1.0 / 1600)
    U = np.stack(ctx.su.interpolate(dg.taylor_green))
    u = torch.from_numpy(U.ravel().copy())
    assert kinetic_energy(ctx, u) == pytest.approx(dg.kinetic_energy(ctx.su, U), rel=1e-14)
    assert kinetic_energy(ctx, 2 * u) == pytest.approx(4 * kinetic_energy(ctx, u), rel=1e-14)
