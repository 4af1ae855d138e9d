"""BDF2 dual-splitting time step (oracle; test infrastructure).

Sec. 3.1 of the paper (four substeps of the dual splitting scheme with BDF
order J = 2 and extrapolation of the convective term) in the matrix form of
Sec. 3.3, with the readings: gamma0 = 3/2, alpha = (2, -1/2), beta = (2, -1)
(the first step BDF1: gamma0 = alpha0 = beta0 = 1); the projection substep
either as the plain L2 projection or with the divergence and continuity
penalty terms (parameters from the extrapolated velocity).
The linear systems are solved exactly with dense factorisations (small
meshes only): the pressure by the eigen-decomposition pseudo-inverse of the
singular periodic Laplacian, the Helmholtz problem by a dense Cholesky solve.
"""
import numpy as np

from . import dg, solvers


class DualSplitting:
    def __init__(self, mesh, ku, nu, dt, penalty_factor=1.0, projection="l2", zeta=(1.0, 1.0)):
        self.su, self.sp = dg.Space(mesh, ku), dg.Space(mesh, ku - 1)
        self.C = dg.Convective(self.su)
        self.M = dg.Mass(self.su)
        self.D = dg.Divergence(self.su, self.sp)
        self.G = dg.Gradient(self.su, self.sp)
        self.nu, self.dt = nu, dt
        self.pf = penalty_factor
        self.projection, self.zeta = projection, zeta
        L = dg.Laplace(self.sp, penalty_factor).matrix()
        w, V = np.linalg.eigh(0.5 * (L + L.T))
        keep = w > 1e-10 * w[-1]
        self.Lpinv = (V[:, keep] / w[keep]) @ V[:, keep].T
        self._H = {}

    def helmholtz_solve(self, mf, B):
        if mf not in self._H:
            H = dg.Helmholtz(self.su, self.nu, mf, self.pf)
            n, E = self.su.size, self.su.mesh.E
            A = np.empty((n, n))
            for j in range(n):
                e = np.zeros(n)
                e[j] = 1.0
                A[:, j] = H.apply(e.reshape(1, E, -1)).ravel()
            self._H[mf] = np.linalg.cholesky(0.5 * (A + A.T))
        Lc = self._H[mf]
        E = self.su.mesh.E
        out = []
        for c in range(3):
            y = np.linalg.solve(Lc, B[c].ravel())
            out.append(np.linalg.solve(Lc.T, y).reshape(E, -1))
        return np.stack(out)

    def step(self, u, u_prev, c_prev, first):
        dt = self.dt
        if first:
            g0, a, b = 1.0, (1.0, 0.0), (1.0, 0.0)
        else:
            g0, a, b = 1.5, (2.0, -0.5), (2.0, -1.0)
        c = self.C.apply(u)
        cc = b[0] * c + (b[1] * c_prev if not first else 0.0)
        hist = a[0] * u + (a[1] * u_prev if not first else 0.0)
        uh = (hist - dt * self.M.apply_inverse(cc)) / g0
        rhs = -(g0 / dt) * self.D.apply(uh)
        p = (self.Lpinv @ rhs.ravel()).reshape(rhs.shape)
        if self.projection == "l2":
            uhh = uh - (dt / g0) * self.M.apply_inverse(self.G.apply(p))
        else:
            # (M + A_D + A_C) uhh = M uh - (dt/gamma0) G p, penalty parameters
            # from the extrapolated velocity (Sec. 3.2), CG with M^-1
            u_ex = u if first else b[0] * u + b[1] * u_prev
            td, tc = dg.penalty_parameters(self.su, u_ex, dt, *self.zeta)
            P = dg.Projection(self.su, td, tc)
            rhs = self.M.apply(uh) - (dt / g0) * self.G.apply(p)
            shape = rhs.shape
            x, _, _ = solvers.pcg(lambda v: P.apply(v.reshape(shape)).ravel(), rhs.ravel(),
                                  precond=lambda r: self.M.apply_inverse(r.reshape(shape)).ravel(),
                                  rel_tol=1e-14, max_iter=200)
            uhh = x.reshape(shape)
        u_new = self.helmholtz_solve(g0 / dt, (g0 / dt) * self.M.apply(uhh))
        return u_new, c

    def run(self, u0, nsteps):
        u, u_prev, c_prev = u0, u0, u0
        for n in range(nsteps):
            u_next, c = self.step(u, u_prev, c_prev, n == 0)
            u_prev, u, c_prev = u, u_next, c
        return u


def _dense(apply, n_in, shape_in):
    """Dense matrix of a linear map given by `apply` (small meshes only)."""
    cols = []
    for j in range(n_in):
        e = np.zeros(n_in)
        e[j] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


class Adjoint:
    """Reverse mode of DualSplitting.run with the plain L2 projection: the
    gradient of J(u^n) with respect to u^0, given dJ/du^n.

    Every substep of Sec. 3.1 is linear in its inputs except the convective
    term, so the backward sweep applies the transposes of the step's linear
    maps (assembled densely: D, G, M^-1, the Helmholtz solve, the
    pseudo-inverse of L) and the convective term's vector-Jacobian product
    (Convective.vjp) at the forward state of each step, in reverse order.
    The carried state of a step is (u^n, u^{n-1}, c^{n-1}); its adjoint is
    propagated through a0 u + a1 u_prev, b0 c + b1 c_prev and c = C(u^n)."""

    def __init__(self, ds):
        if ds.projection != "l2":
            raise ValueError("the adjoint is written for the L2 projection")
        self.ds = ds
        su, sp = ds.su, ds.sp
        E = su.mesh.E
        nu_, np_ = su.size, sp.size
        self.Dm = _dense(lambda v: ds.D.apply(v), 3 * nu_, (3, E, -1))        # (np, 3 nu)
        self.Gm = _dense(lambda v: ds.G.apply(v), np_, (E, -1))               # (3 nu, np)
        self.Minv = _dense(lambda v: ds.M.apply_inverse(v), nu_, (E, -1))     # (nu, nu)
        self.Mm = _dense(lambda v: ds.M.apply(v), nu_, (E, -1))

    def _minv3_T(self, X):
        return np.stack([(self.Minv.T @ X[c].ravel()).reshape(X[c].shape) for c in range(3)])

    def _m3_T(self, X):
        return np.stack([(self.Mm.T @ X[c].ravel()).reshape(X[c].shape) for c in range(3)])

    def gradient(self, u0, nsteps, dJ):
        """u0: initial velocity (3, E, N^3); dJ: callable u^n -> dJ/du^n."""
        ds = self.ds
        dt = ds.dt
        # forward, recording the inputs of every step
        states = []
        u, u_prev, c_prev = u0, u0, u0
        for n in range(nsteps):
            states.append((u, u_prev, c_prev))
            u_next, c = ds.step(u, u_prev, c_prev, n == 0)
            u_prev, u, c_prev = u, u_next, c
        # backward: adjoints of the carried state (u^{n+1}, u^n as u_prev, c^n)
        bu_next = dJ(u)
        bu_cur = np.zeros_like(u0)       # adjoint of u^n through its use as u_prev
        bc_cur = np.zeros_like(u0)       # adjoint of c^n through its use as c_prev
        shape = u0.shape
        for n in reversed(range(nsteps)):
            u, u_prev, c_prev = states[n]
            first = n == 0
            g0, a, b = (1.0, (1.0, 0.0), (1.0, 0.0)) if first else (1.5, (2.0, -0.5), (2.0, -1.0))
            # u_new = H^-1 ((g0/dt) M uhh): H and M symmetric, so the transpose
            # solve is the same solve
            buhh = (g0 / dt) * self._m3_T(ds.helmholtz_solve(g0 / dt, bu_next))
            # uhh = uh - (dt/g0) M^-1 G p
            buh = buhh.copy()
            bp = -(dt / g0) * (self.Gm.T @ self._minv3_T(buhh).ravel())
            # p = L^+ rhs (symmetric pseudo-inverse), rhs = -(g0/dt) D uh
            brhs = ds.Lpinv.T @ bp
            buh += (-(g0 / dt) * (self.Dm.T @ brhs)).reshape(shape)
            # uh = (a0 u + a1 u_prev - dt M^-1 (b0 c + b1 c_prev)) / g0
            bhist = buh / g0
            bcc = -(dt / g0) * self._minv3_T(buh)
            bc = b[0] * bcc + bc_cur             # c = C(u) also leaves as c_prev of step n+1
            bu = a[0] * bhist + ds.C.vjp(u, bc) + bu_cur
            if first:
                # step 0 takes u_prev = c_prev = u^0 but multiplies them by 0
                return bu
            bu_prev = a[1] * bhist
            bc_prev = b[1] * bcc
            bu_next, bu_cur, bc_cur = bu, bu_prev, bc_prev
        return bu_next
