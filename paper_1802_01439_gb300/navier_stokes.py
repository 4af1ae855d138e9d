"""Dual-splitting BDF2 time step of the incompressible Navier-Stokes equations
(Sec. 3.1 and the matrix form of Sec. 3.3 of arXiv:1802.01439), composed of
libdgns operators, with reverse-mode differentiation.

Every operator is a ``torch.autograd.Function`` whose forward and backward
call CUDA kernels of libdgns through the C ABI:

  convective C(u)          backward: the hand-written VJP kernel (dC/du)^T g
  inverse mass / mass      self-adjoint: the forward kernel on g
  divergence D / gradient G    D^T = -G and G^T = -D: the other kernel, negated
  pressure solve L^+ b     self-adjoint: the same FP64 CG + multigrid solve on g
  Helmholtz solve H^-1 b   self-adjoint: the same CG + inverse-mass solve on g
  a x + b y                scaled copies of g
  dissipation eps(u)       its gradient kernel (2 nu / |Omega|) K u

One step (BDF2 with gamma0 = 3/2, alpha = (2, -1/2), beta = (2, -1); the first
step BDF1 with gamma0 = alpha0 = beta0 = 1):
  1. convective:  uh  = (sum_i alpha_i u^{n-i} - dt M^-1 sum_i beta_i C(u^{n-i})) / gamma0
  2. pressure:    L p = -(gamma0/dt) D uh
  3. projection:  uhh = uh - (dt/gamma0) M^-1 G p        (plain L2 projection), or
                  (M + A_D + A_C) uhh = M uh - (dt/gamma0) G p   (penalty terms)
  4. viscous:     (gamma0/dt M + V) u^{n+1} = (gamma0/dt) M uhh
``run`` advances several steps; with ``checkpoint=True`` each step is wrapped
in ``torch.utils.checkpoint`` so only the step inputs are stored and the step
is recomputed during the backward pass.
"""
import torch
from torch.utils.checkpoint import checkpoint


class _Conv(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, u):
        y = torch.empty_like(u)
        dg.vmult_convective(y, u)
        fctx.dg = dg
        fctx.save_for_backward(u)
        return y

    @staticmethod
    def backward(fctx, g):
        (u,) = fctx.saved_tensors
        out = torch.empty_like(u)
        fctx.dg.vjp_convective(out, u, g.contiguous())
        return None, out


class _InvMass(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, x):
        y = torch.empty_like(x)
        dg.apply_inverse_mass(y, x, ncomp=3, space=0)
        fctx.dg = dg
        return y

    @staticmethod
    def backward(fctx, g):
        out = torch.empty_like(g)
        fctx.dg.apply_inverse_mass(out, g.contiguous(), ncomp=3, space=0)
        return None, out


class _Mass(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, x):
        y = torch.empty_like(x)
        dg.vmult_mass(y, x, ncomp=3, space=0)
        fctx.dg = dg
        return y

    @staticmethod
    def backward(fctx, g):
        out = torch.empty_like(g)
        fctx.dg.vmult_mass(out, g.contiguous(), ncomp=3, space=0)
        return None, out


class _Div(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, u):
        y = torch.empty(dg.n_p, dtype=u.dtype, device=u.device)
        dg.vmult_divergence(y, u)
        fctx.dg = dg
        return y

    @staticmethod
    def backward(fctx, g):
        dg = fctx.dg
        out = torch.empty(3 * dg.n_u, dtype=g.dtype, device=g.device)
        dg.vmult_gradient(out, g.contiguous())      # D^T = -G
        dg.axpby(out, out, 0.0, -1.0)
        return None, out


class _Grad(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, p):
        y = torch.empty(3 * dg.n_u, dtype=p.dtype, device=p.device)
        dg.vmult_gradient(y, p)
        fctx.dg = dg
        return y

    @staticmethod
    def backward(fctx, g):
        dg = fctx.dg
        out = torch.empty(dg.n_p, dtype=g.dtype, device=g.device)
        dg.vmult_divergence(out, g.contiguous())    # G^T = -D
        dg.axpby(out, out, 0.0, -1.0)
        return None, out


def _solve_start(b, x0):
    """The solution vector of a solve: x0 (a detached copy) when an initial
    guess is given, else zeros."""
    if x0 is None:
        return torch.zeros_like(b), 0
    return x0.detach().clone().contiguous(), 1


class _Poisson(torch.autograd.Function):
    """x = L^+ b: the zero-mean solution of the periodic pressure problem.
    opts: solve parameters (rel_tol, abs_tol); log: a list the solve info is
    appended to (or None); x0: an initial guess (not differentiated)."""

    @staticmethod
    def forward(fctx, dg, b, opts, log, x0=None):
        x, guess = _solve_start(b, x0)
        info = dg.cg_mg_solve(x, b.contiguous(), use_initial_guess=guess, **opts)
        if log is not None:
            log.append(("pressure", info))
        fctx.dg, fctx.opts = dg, opts
        return x

    @staticmethod
    def backward(fctx, g):
        x = torch.zeros_like(g)
        fctx.dg.cg_mg_solve(x, g.contiguous(), **fctx.opts)
        return None, x, None, None, None


class _Helmholtz(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, b, mass_factor, opts, log, x0=None):
        x, guess = _solve_start(b, x0)
        info = dg.cg_invmass_solve(x, b.contiguous(), mass_factor, use_initial_guess=guess, **opts)
        if log is not None:
            log.append(("viscous", info))
        fctx.dg, fctx.mf, fctx.opts = dg, mass_factor, opts
        return x

    @staticmethod
    def backward(fctx, g):
        x = torch.zeros_like(g)
        fctx.dg.cg_invmass_solve(x, g.contiguous(), fctx.mf, **fctx.opts)
        return None, x, None, None, None, None


class _Projection(torch.autograd.Function):
    """x = (M + A_D + A_C)^-1 b with the penalty parameters held fixed."""

    @staticmethod
    def forward(fctx, dg, b, tau_d, tau_c, opts, log, x0=None):
        x, guess = _solve_start(b, x0)
        info = dg.cg_projection_solve(x, b.contiguous(), tau_d, tau_c, use_initial_guess=guess, **opts)
        if log is not None:
            log.append(("projection", info))
        fctx.dg, fctx.opts = dg, opts
        fctx.save_for_backward(tau_d, tau_c)
        return x

    @staticmethod
    def backward(fctx, g):
        tau_d, tau_c = fctx.saved_tensors
        x = torch.zeros_like(g)
        fctx.dg.cg_projection_solve(x, g.contiguous(), tau_d, tau_c, **fctx.opts)
        return None, x, None, None, None, None, None


class _Axpby(torch.autograd.Function):
    """a x + b y (a new tensor)."""

    @staticmethod
    def forward(fctx, dg, x, y, a, b):
        z = y.clone() if b != 0.0 else torch.empty_like(y)
        dg.axpby(z, x.contiguous(), a, b)
        fctx.dg, fctx.a, fctx.b = dg, a, b
        return z

    @staticmethod
    def backward(fctx, g):
        g = g.contiguous()
        gx = torch.empty_like(g)
        fctx.dg.axpby(gx, g, fctx.a, 0.0)
        gy = torch.empty_like(g)
        fctx.dg.axpby(gy, g, fctx.b, 0.0)
        return None, gx, gy, None, None


class _Dissipation(torch.autograd.Function):
    @staticmethod
    def forward(fctx, dg, u):
        fctx.dg = dg
        fctx.save_for_backward(u)
        return torch.tensor(dg.dissipation(u), dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(fctx, g):
        (u,) = fctx.saved_tensors
        out = torch.empty_like(u)
        fctx.dg.dissipation_grad(out, u)
        fctx.dg.axpby(out, out, 0.0, float(g))
        return None, out


def lincomb(dg, a, x, b, y):
    return _Axpby.apply(dg, x, y, float(a), float(b))


def _extrapolate(dg, hist):
    """Second-order extrapolation 2 h[-1] - h[-2] of a solution history (the
    last entry alone when only one exists); detached."""
    if len(hist) == 1:
        return hist[-1]
    out = torch.empty_like(hist[-1])
    dg.axpby(out, hist[-1], 2.0, 0.0)
    dg.axpby(out, hist[-2], -1.0, 1.0)
    return out


class DualSplitting:
    """BDF2 dual-splitting stepper on a libdgns ``Context`` (velocity degree
    k_u, pressure degree k_p = k_u - 1, FP32 or FP64 multigrid)."""

    def __init__(self, dg, dt, solver_tol=1e-12, projection="l2", zeta_d=1.0, zeta_c=1.0, abs_tol=0.0,
                 guess="zero"):
        """projection: "l2" (plain L2 projection) or "penalty" (the
        divergence and continuity penalty terms of Sec. 3.2 with factors
        zeta_d, zeta_c; the penalty parameters come from the extrapolated
        velocity and are treated as constants by the reverse mode).
        solver_tol, abs_tol: relative (to the initial residual) and absolute
        tolerance of the three CG solves (the paper's runs: 1e-6, 1e-12).
        guess: "zero" or "extrapolate" (initial guesses of the pressure,
        projection and viscous solves extrapolated from the previous steps,
        Sec. 3.3)."""
        if projection not in ("l2", "penalty"):
            raise ValueError(projection)
        if guess not in ("zero", "extrapolate"):
            raise ValueError(guess)
        self.dg = dg
        self.dt = float(dt)
        self.tol = float(solver_tol)
        self.opts = {"rel_tol": float(solver_tol), "abs_tol": float(abs_tol)}
        self.projection = projection
        self.zeta = (float(zeta_d), float(zeta_c))
        self.guess = guess
        self.log = None   # set to a list to collect (substep, solve info) pairs

    def coefficients(self, first):
        if first:
            return 1.0, (1.0, 0.0), (1.0, 0.0)
        return 1.5, (2.0, -0.5), (2.0, -1.0)

    def step(self, u, u_prev, c_prev, first, guesses=None):
        """Returns (u^{n+1}, C(u^n), p^{n+1}, uhh) -- the last two detached,
        for the extrapolation of initial guesses.  guesses: None or initial
        guesses (pressure, projected velocity, new velocity) of the solves."""
        dg, dt, opts, log = self.dg, self.dt, self.opts, self.log
        g0, a, b = self.coefficients(first)
        gp, gq, gu = guesses if guesses is not None else (None, None, None)
        c = _Conv.apply(dg, u)
        cc = c if first else lincomb(dg, b[0], c, b[1], c_prev)
        hist = u if first else lincomb(dg, a[0], u, a[1], u_prev)
        uh = lincomb(dg, -dt / g0, _InvMass.apply(dg, cc), 1.0 / g0, hist)
        rhs = _Div.apply(dg, uh)
        p = _Poisson.apply(dg, lincomb(dg, 0.0, rhs, -g0 / dt, rhs), opts, log, gp)
        if self.projection == "l2":
            uhh = lincomb(dg, -dt / g0, _InvMass.apply(dg, _Grad.apply(dg, p)), 1.0, uh)
        else:
            with torch.no_grad():
                u_ex = u if first else lincomb(dg, b[0], u, b[1], u_prev)
                tau_d, tau_c = dg.penalty_parameters(u_ex.detach().contiguous(), dt, *self.zeta)
            rhs_p = lincomb(dg, -dt / g0, _Grad.apply(dg, p), 1.0, _Mass.apply(dg, uh))
            uhh = _Projection.apply(dg, rhs_p, tau_d, tau_c, opts, log, gq)
        bh = lincomb(dg, 0.0, uhh, g0 / dt, _Mass.apply(dg, uhh))
        u_new = _Helmholtz.apply(dg, bh, g0 / dt, opts, log, gu)
        return u_new, c, p.detach(), uhh.detach()

    def run(self, u0, nsteps, checkpoint_steps=True, callback=None):
        """Advance nsteps from u0; returns the final velocity.  callback(n, u)
        (if given) sees the velocity after every step n = 1..nsteps."""
        u, u_prev, c_prev = u0, u0, u0
        hp, hq, hu = [], [], [u0.detach()]
        for n in range(nsteps):
            first = n == 0
            guesses = None
            if self.guess == "extrapolate":
                with torch.no_grad():
                    guesses = (_extrapolate(self.dg, hp) if hp else None,
                               _extrapolate(self.dg, hq) if hq else None,
                               _extrapolate(self.dg, hu))
            if checkpoint_steps and torch.is_grad_enabled():
                u_next, c, p, uhh = checkpoint(self.step, u, u_prev, c_prev, first, guesses, use_reentrant=False)
            else:
                u_next, c, p, uhh = self.step(u, u_prev, c_prev, first, guesses)
            u_prev, u, c_prev = u, u_next, c
            if self.guess == "extrapolate":
                hp, hq, hu = (hp + [p])[-2:], (hq + [uhh])[-2:], (hu + [u.detach()])[-2:]
            if callback is not None:
                callback(n + 1, u)
        return u

    def dissipation(self, u):
        return _Dissipation.apply(self.dg, u)
