"""Host orchestration of the BDF2 stepper and its autograd Functions
(paper_1802_01439_gb300/navier_stokes.py) on the CPU, driven through the
oracle-backed test double of tests/host_double.py (exact dense solves):

  * the product stepper's substeps, coefficients and signs reproduce the
    oracle's own dual-splitting step (L2 and penalty projection);
  * extrapolated initial guesses leave the result unchanged when the solves
    are exact;
  * every autograd Function passes gradcheck (the transposes and
    self-adjoint reuses of the backward pass);
  * the gradient of eps(u^n) through checkpointed steps matches central
    differences.
The same stepper on the CUDA library is tested in tests/test_gpu_timestep.py.
"""
import numpy as np
import pytest
import torch

from oracle import dg, timestep
from paper_1802_01439_gb300 import navier_stokes as ns
from tests.host_double import OracleContext


def _field(s, seed, noise=1e-2):
    m = s.mesh
    u = np.stack(s.interpolate(dg.taylor_green))
    return u + noise * np.random.default_rng(seed).uniform(-1, 1, (3, m.E, s.ndofs_cell))


@pytest.mark.parametrize("projection", ["l2", "penalty"])
def test_stepper_reproduces_the_oracle_step(projection):
    m, k, nu, dt = dg.Mesh((2, 2, 1)), 3, 1.0 / 1600, 1e-3
    ctx = OracleContext(m, k, nu)
    u0 = _field(ctx.su, 4)
    stepper = ns.DualSplitting(ctx, dt, projection=projection)
    with torch.no_grad():
        u = stepper.run(torch.from_numpy(u0.ravel().copy()), 3).numpy()
    ref = timestep.DualSplitting(m, k, nu, dt, projection=projection).run(u0, 3)
    assert np.max(np.abs(u - ref.ravel())) <= 1e-11 * np.max(np.abs(ref))


def test_extrapolated_guesses_keep_the_result():
    m, k, nu, dt = dg.Mesh((2, 1, 2)), 2, 0.01, 1e-2
    ctx = OracleContext(m, k, nu)
    u0 = torch.from_numpy(_field(ctx.su, 5).ravel().copy())
    with torch.no_grad():
        a = ns.DualSplitting(ctx, dt, projection="penalty").run(u0, 4)
        b = ns.DualSplitting(ctx, dt, projection="penalty", guess="extrapolate").run(u0, 4)
    assert torch.max(torch.abs(a - b)) <= 1e-11 * torch.max(torch.abs(a))


def test_autograd_functions_gradcheck():
    m, k = dg.Mesh((1, 2, 1)), 2
    ctx = OracleContext(m, k, 0.05)
    rng = np.random.default_rng(6)
    u = torch.from_numpy(_field(ctx.su, 7, 1e-1).ravel().copy()).requires_grad_()
    p = torch.from_numpy(rng.uniform(-1, 1, ctx.n_p)).requires_grad_()
    kw = dict(eps=1e-6, atol=1e-7, rtol=1e-6)
    opts = {"rel_tol": 1e-13, "abs_tol": 0.0}
    assert torch.autograd.gradcheck(lambda x: ns._Conv.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._InvMass.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Mass.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Div.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Grad.apply(ctx, x), (p,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Helmholtz.apply(ctx, x, 100.0, opts, None), (u,), **kw)
    td, tc = ctx.penalty_parameters(u.detach(), 1e-2)
    assert torch.autograd.gradcheck(lambda x: ns._Projection.apply(ctx, x, td, tc, opts, None), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x, y: ns.lincomb(ctx, 0.3, x, -1.7, y), (u, u.detach().clone().requires_grad_()), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Dissipation.apply(ctx, x), (u,), **kw)
    pm = (p - p.mean()).detach().requires_grad_()
    assert torch.autograd.gradcheck(lambda x: ns._Poisson.apply(ctx, x - x.mean(), opts, None), (pm,), **kw)


def test_checkpointed_gradient_matches_central_differences():
    """J = eps(u^2) after two steps; <grad J, v> against the central
    difference along seeded directions.  A uniform offset keeps the normal
    velocities away from the LLF kinks, so the quotient is smooth."""
    m, k, nu, dt = dg.Mesh((2, 1, 1)), 2, 0.02, 1e-2
    ctx = OracleContext(m, k, nu)
    stepper = ns.DualSplitting(ctx, dt, solver_tol=1e-13)
    u0 = torch.from_numpy(_field(ctx.su, 8).ravel().copy() + 0.3)
    x = u0.clone().requires_grad_()
    J = stepper.dissipation(stepper.run(x, 2))
    J.backward()
    delta = 1e-6
    for seed in (1, 2):
        v = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, u0.numel()))
        with torch.no_grad():
            jp = float(stepper.dissipation(stepper.run(u0 + delta * v, 2, checkpoint_steps=False)))
            jm = float(stepper.dissipation(stepper.run(u0 - delta * v, 2, checkpoint_steps=False)))
        fd = (jp - jm) / (2 * delta)
        ad = float(torch.dot(x.grad, v))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
