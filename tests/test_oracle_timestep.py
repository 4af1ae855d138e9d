"""Pins of the oracle's dual-splitting BDF2 step (no GPU).

  * a constant velocity is a steady state (C(const) = 0, D const = 0,
    V const = 0, so every substep returns its input);
  * the pressure projection removes most of the discrete divergence of a
    perturbed Taylor-Green field;
  * halving dt moves the result towards a fine-dt reference (consistency of
    the time stepping).
"""
import numpy as np

from oracle import dg, timestep


def test_constant_velocity_is_steady():
    m = dg.Mesh((2, 2, 2))
    ts = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3)
    s = ts.su
    u0 = np.stack([np.full((m.E, s.ndofs_cell), v) for v in (0.3, -0.2, 0.1)])
    u = ts.run(u0, 3)
    assert np.max(np.abs(u - u0)) < 1e-11


def test_projection_reduces_divergence():
    m = dg.Mesh((3, 3, 3))
    ts = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3)
    s = ts.su
    u0 = np.stack(s.interpolate(dg.taylor_green)) + 1e-2 * np.random.default_rng(0).uniform(-1, 1, (3, m.E, s.ndofs_cell))
    u1 = ts.run(u0, 1)
    assert np.linalg.norm(ts.D.apply(u1)) < 0.2 * np.linalg.norm(ts.D.apply(u0))


def test_time_consistency():
    m = dg.Mesh((2, 2, 2))
    nu = 0.05
    s = dg.Space(m, 3)
    u0 = np.stack(s.interpolate(dg.taylor_green))
    big = timestep.DualSplitting(m, 3, nu, 2e-3).run(u0, 2)
    small = timestep.DualSplitting(m, 3, nu, 1e-3).run(u0, 4)
    tiny = timestep.DualSplitting(m, 3, nu, 5e-4).run(u0, 8)
    e1 = np.max(np.abs(big - tiny))
    e2 = np.max(np.abs(small - tiny))
    assert e2 < 0.6 * e1


def test_penalty_projection_zero_factors_is_l2_projection():
    # with zeta_D = zeta_C = 0 the penalty operator is M, so the projection
    # substep (M) uhh = M uh - dt/gamma0 G p is the plain L2 projection
    m = dg.Mesh((2, 2, 2))
    s = dg.Space(m, 3)
    u0 = np.stack(s.interpolate(dg.taylor_green)) + 1e-2 * np.random.default_rng(1).uniform(-1, 1, (3, m.E, s.ndofs_cell))
    a = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3).run(u0, 2)
    b = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3, projection="penalty", zeta=(0.0, 0.0)).run(u0, 2)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_penalty_projection_keeps_constants_and_lowers_divergence():
    m = dg.Mesh((2, 2, 2))
    ts = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3, projection="penalty")
    s = ts.su
    u0 = np.stack([np.full((m.E, s.ndofs_cell), v) for v in (0.3, -0.2, 0.1)])
    assert np.max(np.abs(ts.run(u0, 3) - u0)) < 1e-11
    m = dg.Mesh((3, 3, 3))
    s = dg.Space(m, 3)
    u0 = np.stack(s.interpolate(dg.taylor_green)) + 1e-2 * np.random.default_rng(0).uniform(-1, 1, (3, m.E, s.ndofs_cell))
    l2 = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3)
    pen = timestep.DualSplitting(m, 3, 1.0 / 1600, 1e-3, projection="penalty", zeta=(10.0, 10.0))
    assert np.linalg.norm(l2.D.apply(pen.run(u0, 1))) < np.linalg.norm(l2.D.apply(l2.run(u0, 1)))
