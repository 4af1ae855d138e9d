"""GPU parity of the differentiated dual-splitting path: the convective VJP
kernel, the dissipation functional and its gradient, the BDF2 step against
the oracle's step, autograd gradients of every operator (gradcheck), and the
gradient of the final dissipation rate after BDF2 steps against central
finite differences (the 20-step, 32^3, k=4 Taylor-Green case included),
and the two-dimensional Taylor-Green vortex (an exact solution) reproduced
by the GPU stepper.
"""
import numpy as np
import pytest
import torch

from oracle import dg, rules, timestep
from paper_1802_01439_gb300 import inputs
from tests.gpu_common import build_lib, context, dev, host, random_field, rel_err, tgv_field

OPTS = {"rel_tol": 1e-13, "abs_tol": 0.0}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,k,field", [((3, 2, 2), 3, "tgv"), ((2, 2, 3), 2, "rand"), ((1, 2, 1), 4, "rand"),
                                       ((2, 1, 2), 7, "tgv"), ((2, 2, 2), 1, "rand"), ((3, 3, 1), 5, "tgv")])
def test_convective_vjp(n, k, field, mode):
    """mode 0: native FP64; mode 1: double-float arithmetic."""
    ctx = context(n, k, max(k - 1, 1), mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-3, 0) if field == "tgv" else random_field(s, 3, 1)
    w = random_field(s, 3, 2)
    g = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vjp_convective(g, dev(u), dev(w))
    assert rel_err(host(g), dg.Convective(s).vjp(u, w)) <= 1e-12


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,k,nq", [((1, 2, 1), 8, 0), ((2, 1, 1), 9, 0), ((1, 1, 2), 10, 0), ((1, 2, 1), 11, 0),
                                    ((2, 1, 1), 9, 10), ((1, 1, 2), 11, 12)])
def test_convective_vjp_high_degree(n, k, nq, mode):
    """k = 8..11: the kernel contracts plane by plane (z first); over-integrated
    (nq = 0: 3(k+1)/2 points) and with k + 1 points."""
    ctx = context(n, k, k - 1, mg_precision=0, fp64_mode=mode, n_q_conv=nq)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-3, 0) if k % 2 else random_field(s, 3, 4)
    w = random_field(s, 3, 5)
    g = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vjp_convective(g, dev(u), dev(w))
    C = dg.Convective(s, nq=nq if nq else None)
    assert rel_err(host(g), C.vjp(u, w)) <= 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_dissipation_and_gradient(mode):
    nu = 1.0 / 1600
    n, k = (3, 2, 4), 4
    ctx = context(n, k, mg_precision=0, nu=nu, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-2, 3)
    eps = ctx.dissipation(dev(u))
    ref = dg.dissipation_rate(s, u, nu)
    assert abs(eps - ref) <= 1e-12 * abs(ref)
    g = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.dissipation_grad(g, dev(u))
    assert rel_err(host(g), dg.dissipation_gradient(s, u, nu)) <= 1e-12


def _stepper(n, k, nu, dt, prec=32):
    from paper_1802_01439_gb300.navier_stokes import DualSplitting
    ctx = context(n, k, k - 1, mg_precision=prec, nu=nu)
    return ctx, DualSplitting(ctx, dt, solver_tol=1e-13)


def test_bdf2_steps_match_oracle():
    n, k, nu, dt = (4, 2, 2), 3, 1.0 / 1600, 1e-3
    ctx, ds = _stepper(n, k, nu, dt)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    u0 = tgv_field(s, 1e-2, 4)
    with torch.no_grad():
        u = ds.run(dev(u0.ravel()), 3)
    ref = timestep.DualSplitting(m, k, nu, dt).run(u0, 3)
    # dense exact solves in the oracle vs CG to 1e-13 here
    assert rel_err(host(u), ref) <= 1e-9


def test_operator_gradients_gradcheck():
    from paper_1802_01439_gb300 import navier_stokes as ns
    n, k = (2, 1, 2), 2
    ctx, ds = _stepper(n, k, 0.05, 1e-2, prec=64)
    s = dg.Space(dg.Mesh(n), k)
    u = dev(tgv_field(s, 1e-1, 5).ravel()).requires_grad_()
    p = dev(np.random.default_rng(6).uniform(-1, 1, ctx.n_p)).requires_grad_()
    kw = dict(eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)
    assert torch.autograd.gradcheck(lambda x: ns._Conv.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._InvMass.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Mass.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Div.apply(ctx, x), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Grad.apply(ctx, x), (p,), **kw)
    assert torch.autograd.gradcheck(lambda x: ns._Helmholtz.apply(ctx, x, 100.0, OPTS, None), (u,), **kw)
    assert torch.autograd.gradcheck(lambda x: ds.dissipation(x), (u,), **kw)
    pm = (p - p.mean()).detach().requires_grad_()
    assert torch.autograd.gradcheck(lambda x: ns._Poisson.apply(ctx, x - x.mean(), OPTS, None), (pm,), **kw)


@pytest.mark.parametrize("n,k,steps", [((2, 2, 1), 2, 3), ((3, 1, 2), 3, 2)])
def test_gradient_matches_oracle_adjoint(n, k, steps):
    """The GPU's checkpointed reverse mode (hand-written VJP kernels, adjoint
    solves) against the oracle's adjoint of the same BDF2 steps (dense
    transposes of every linear map, Convective.vjp): the whole gradient of
    eps(u^n) w.r.t. u^0, elementwise.  The GPU solves with CG to 1e-13, the
    oracle exactly."""
    nu, dt = 1.0 / 1600, 1e-3
    ctx, ds = _stepper(n, k, nu, dt)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    u0 = tgv_field(s, 1e-2, 0)
    x = dev(u0.ravel()).requires_grad_()
    ds.dissipation(ds.run(x, steps)).backward()
    ods = timestep.DualSplitting(m, k, nu, dt)
    ref = timestep.Adjoint(ods).gradient(u0, steps, lambda u: dg.dissipation_gradient(s, u, nu))
    assert rel_err(host(x.grad), ref) <= 1e-9


def _fd_check(n, k, nu, dt, steps, ndir, delta, tol, noise=1e-3, offset=0.0):
    """Central differences of J = eps(u^steps) along seeded directions against
    <grad J, v> from autograd.  J is only piecewise smooth: the LLF flux has
    kinks at u.n = 0 and at |u-.n| = |u+.n|, and a finite step crosses some of
    them, so the difference quotient differs from the one-sided derivative by
    O(delta); the tolerance is set for the step used (the error was measured
    to fall linearly with delta)."""
    ctx, ds = _stepper(n, k, nu, dt)
    s = dg.Space(dg.Mesh(n), k)
    u0 = dev(tgv_field(s, noise, 0).ravel() + offset)
    x = u0.clone().requires_grad_()
    J = ds.dissipation(ds.run(x, steps))
    J.backward()
    grad = x.grad.detach()
    worst = 0.0
    with torch.no_grad():
        for d in range(1, ndir + 1):
            v = dev(np.random.default_rng(d).uniform(-1, 1, u0.numel()))
            jp = ds.dissipation(ds.run(u0 + delta * v, steps, checkpoint_steps=False))
            jm = ds.dissipation(ds.run(u0 - delta * v, steps, checkpoint_steps=False))
            fd = (float(jp) - float(jm)) / (2 * delta)
            ad = float(torch.dot(grad, v))
            worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= tol, worst
    return worst


def test_gradient_small_fd():
    _fd_check((4, 2, 2), 3, 1.0 / 1600, 1e-3, 3, 4, 1e-6, 1e-6)


def test_gradient_small_fd_without_kinks_nearby():
    """A uniform offset keeps every normal velocity away from zero: the
    difference quotient then matches to 1e-7."""
    _fd_check((4, 2, 2), 3, 1.0 / 1600, 1e-3, 3, 3, 1e-6, 1e-7, noise=0.0, offset=0.3)


@pytest.mark.slow
def test_gradient_taylor_green_32c_k4_20_steps():
    """The differentiated-solver workload: 32^3 cells, k_u = 4, dt = 1e-3,
    Re = 1600, 20 BDF2 steps, gradient of eps(u^20) w.r.t. u^0 along 8 seeded
    directions (measured worst error 8e-6 at delta = 1e-7, falling linearly
    with delta)."""
    _fd_check(32, 4, 1.0 / 1600, 1e-3, 20, 8, 1e-7, 2e-5)


def test_bdf2_penalty_projection_matches_oracle():
    from paper_1802_01439_gb300.navier_stokes import DualSplitting
    n, k, nu, dt = (4, 2, 2), 3, 1.0 / 1600, 1e-3
    ctx = context(n, k, k - 1, mg_precision=32, nu=nu)
    ds = DualSplitting(ctx, dt, solver_tol=1e-13, projection="penalty")
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    u0 = tgv_field(s, 1e-2, 4)
    with torch.no_grad():
        u = ds.run(dev(u0.ravel()), 3)
    ref = timestep.DualSplitting(m, k, nu, dt, projection="penalty").run(u0, 3)
    assert rel_err(host(u), ref) <= 1e-9


def test_projection_solve_gradcheck():
    from paper_1802_01439_gb300 import navier_stokes as ns
    n, k = (2, 1, 2), 2
    ctx, _ = _stepper(n, k, 0.05, 1e-2, prec=64)
    s = dg.Space(dg.Mesh(n), k)
    u = dev(tgv_field(s, 1e-1, 5).ravel())
    td, tc = ctx.penalty_parameters(u, 0.1, 1.0, 1.0)
    x = u.clone().requires_grad_()
    kw = dict(eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)
    assert torch.autograd.gradcheck(lambda y: ns._Projection.apply(ctx, y, td, tc, OPTS, None), (x,), **kw)


@pytest.mark.parametrize("which", ["mg", "invmass", "projection"])
def test_initial_guess(which):
    """A solve started from an initial guess reaches the same solution as one
    from zero; the relative criterion is taken against the initial residual;
    the exact solution as initial guess stops after one iteration."""
    n, k = (3, 2, 2), 3
    ctx = context(n, k, k - 1, mg_precision=32, nu=0.05)
    s = dg.Space(dg.Mesh(n), k)
    if which == "mg":
        b = dev(random_field(dg.Space(s.mesh, k - 1), 1, 3).ravel())
        b -= b.mean()
        solve = lambda x, **kw: ctx.cg_mg_solve(x, b, **kw)
    elif which == "invmass":
        b = dev(random_field(s, 3, 3).ravel())
        solve = lambda x, **kw: ctx.cg_invmass_solve(x, b, 150.0, **kw)
    else:
        b = dev(random_field(s, 3, 3).ravel())
        td, tc = ctx.penalty_parameters(dev(tgv_field(s, 1e-2, 1).ravel()), 0.1)
        solve = lambda x, **kw: ctx.cg_projection_solve(x, b, td, tc, **kw)
    x0 = torch.zeros_like(b)
    i0 = solve(x0, rel_tol=1e-13)
    xg = dev(np.random.default_rng(9).uniform(-1, 1, b.numel()))
    if which == "mg":
        xg -= xg.mean()
    x1 = xg.clone()
    i1 = solve(x1, rel_tol=1e-13, use_initial_guess=1)
    assert i1["initial_res"] != i0["initial_res"]
    assert rel_err(host(x1), host(x0)) <= 1e-10
    # exact solution as the guess: the absolute criterion stops the solve
    x2 = x0.clone()
    i2 = solve(x2, rel_tol=1e-6, abs_tol=1e-9 * i0["initial_res"], use_initial_guess=1)
    assert i2["iterations"] == 1 and i2["initial_res"] <= 1e-9 * i0["initial_res"]
    assert rel_err(host(x2), host(x0)) <= 1e-11


def test_extrapolated_guesses_accuracy():
    """The paper's solver setting (abs 1e-12, rel 1e-6 to the initial residual)
    with extrapolated and with zero initial guesses, against a run solved to
    1e-13: both stay within the tolerance's reach of the reference, and the
    extrapolated guesses end more accurate (their initial residual is
    smaller, so the same relative reduction ends at a smaller residual)."""
    from paper_1802_01439_gb300.navier_stokes import DualSplitting
    n, k, nu, dt = (4, 4, 4), 3, 1.0 / 1600, 2e-3
    ctx = context(n, k, k - 1, mg_precision=32, nu=nu)
    s = dg.Space(dg.Mesh(n), k)
    u0 = dev(tgv_field(s, 1e-3, 2).ravel())
    out = {}
    for name, tol, guess in (("ref", 1e-13, "zero"), ("zero", 1e-6, "zero"), ("extrapolate", 1e-6, "extrapolate")):
        ds = DualSplitting(ctx, dt, solver_tol=tol, abs_tol=1e-12, projection="penalty", guess=guess)
        ds.log = []
        with torch.no_grad():
            u = ds.run(u0, 6, checkpoint_steps=False)
        assert all(i["status"] == 0 for _, i in ds.log)
        out[name] = host(u)
    err_zero = rel_err(out["zero"], out["ref"])
    err_ex = rel_err(out["extrapolate"], out["ref"])
    assert err_zero <= 1e-4 and err_ex <= 1e-5 and err_ex < err_zero


@pytest.mark.parametrize("mode", [0, 1])
def test_two_dimensional_taylor_green_exact_solution(mode):
    """The GPU stepper reproduces the two-dimensional Taylor-Green vortex
    u = (sin x cos y, -cos x sin y, 0) exp(-2 nu t), an exact Navier-Stokes
    solution: on 4 x 4 x 1 cells, k_u = 4, ten steps of dt = 0.01 at
    nu = 0.1, the max-norm error against the exact field stays within the
    spatial error of the discretisation (1.16e-3 for the oracle's step) and
    the kinetic energy u^T M u follows exp(-4 nu t) to 1e-4 (5e-6 for the
    oracle's step); native FP64 (mode 0) and double-float (mode 1)."""
    from paper_1802_01439_gb300.navier_stokes import DualSplitting
    nu, dt, steps, k, n = 0.1, 0.01, 10, 4, (4, 4, 1)
    ctx = context(n, k, k - 1, nu=nu, fp64_mode=mode)
    ds = DualSplitting(ctx, dt, solver_tol=1e-13)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    X = inputs.node_coordinates(m.n, m.lo, m.hi, rules.lgl_nodes(k))
    u0 = np.stack([np.sin(X[0]) * np.cos(X[1]), -np.cos(X[0]) * np.sin(X[1]), np.zeros_like(X[0])])
    with torch.no_grad():
        u = host(ds.run(dev(u0.ravel()), steps)).reshape(u0.shape)
    t = dt * steps
    assert np.max(np.abs(u - u0 * np.exp(-2 * nu * t))) < 2e-3
    M = dg.Mass(s)
    energy = [sum(np.sum(v[c] * M.apply(v[c:c + 1])[0]) for c in range(3)) for v in (u0, u)]
    assert abs(energy[1] / energy[0] / np.exp(-4 * nu * t) - 1) < 1e-4
