"""A CPU test double of the libdgns Context methods that the time stepper
(paper_1802_01439_gb300/navier_stokes.py) calls, computed by the oracle with
exact dense solves.

Test infrastructure only: it lets the CPU suite exercise the stepper's host
orchestration and its autograd Functions (substep order, BDF coefficients,
signs, the transposes used in the backward pass, extrapolated guesses,
checkpointing) without a GPU.  The product path never uses it; the same
stepper on the CUDA library is compared with the oracle in
tests/test_gpu_timestep.py.
"""
import numpy as np
import torch

from oracle import dg, solvers, timestep


class OracleContext:
    def __init__(self, mesh, ku, nu, penalty_factor=1.0):
        # the oracle's step object holds every operator and the dense solvers;
        # its own time step is not used here
        self._ts = timestep.DualSplitting(mesh, ku, nu, 1.0, penalty_factor)
        self.su, self.sp = self._ts.su, self._ts.sp
        self.nu = nu
        self.n_u, self.n_p = self.su.size, self.sp.size
        self._E = mesh.E

    # ------------------------------------------------------------ helpers
    def _u(self, t):
        return t.detach().numpy().reshape(3, self._E, -1)

    def _p(self, t):
        return t.detach().numpy().reshape(self._E, -1)

    @staticmethod
    def _put(dst, a):
        dst.copy_(torch.from_numpy(np.ascontiguousarray(a).ravel()))
        return dst

    @staticmethod
    def _info():
        return {"rc": 0, "iterations": 0, "rel_res": 0.0}

    # ---------------------------------------------------------- operators
    def vmult_convective(self, dst3, u3):
        return self._put(dst3, self._ts.C.apply(self._u(u3)))

    def vjp_convective(self, grad_u3, u3, w3):
        return self._put(grad_u3, self._ts.C.vjp(self._u(u3), self._u(w3)))

    def vmult_mass(self, dst, src, ncomp=1, space=0):
        assert ncomp == 3 and space == 0
        return self._put(dst, self._ts.M.apply(self._u(src)))

    def apply_inverse_mass(self, dst, src, ncomp=1, space=0):
        assert ncomp == 3 and space == 0
        return self._put(dst, self._ts.M.apply_inverse(self._u(src)))

    def vmult_divergence(self, dst_p, u3):
        return self._put(dst_p, self._ts.D.apply(self._u(u3)))

    def vmult_gradient(self, dst3, p):
        return self._put(dst3, self._ts.G.apply(self._p(p)))

    def axpby(self, y, x, a, b):
        z = a * x if b == 0.0 else a * x + b * y
        y.copy_(z)
        return y

    def dot(self, a, b):
        return float(torch.dot(a, b))

    def dissipation(self, u3):
        return dg.dissipation_rate(self.su, self._u(u3), self.nu)

    def dissipation_grad(self, grad3, u3):
        return self._put(grad3, dg.dissipation_gradient(self.su, self._u(u3), self.nu))

    def penalty_parameters(self, u_ex3, dt, zeta_d=1.0, zeta_c=1.0):
        td, tc = dg.penalty_parameters(self.su, self._u(u_ex3), dt, zeta_d, zeta_c)
        return torch.from_numpy(td), torch.from_numpy(tc)

    # ------------------------------------------------------------- solves
    def cg_mg_solve(self, x, b, raise_on_error=True, **kw):
        self._put(x, self._ts.Lpinv @ b.detach().numpy())
        return self._info()

    def cg_invmass_solve(self, x3, b3, mass_factor, raise_on_error=True, **kw):
        self._put(x3, self._ts.helmholtz_solve(mass_factor, self._u(b3)))
        return self._info()

    def cg_projection_solve(self, x3, b3, tau_d, tau_c, raise_on_error=True, **kw):
        if not torch.any(b3):                      # the library's CG returns x = 0 for b = 0
            x3.zero_()
            return self._info()
        P = dg.Projection(self.su, tau_d.numpy(), tau_c.numpy())
        shape = (3, self._E, -1)
        sol, _, _ = solvers.pcg(lambda v: P.apply(v.reshape(shape)).ravel(), b3.detach().numpy(),
                                precond=lambda r: self._ts.M.apply_inverse(r.reshape(shape)).ravel(),
                                rel_tol=1e-14, max_iter=500)
        self._put(x3, sol)
        return self._info()
