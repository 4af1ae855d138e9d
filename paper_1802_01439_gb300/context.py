"""Python binding of libdgns: a thin wrapper that checks tensor shapes and
dtypes and passes raw pointers to the C ABI (include/dgns.h).  PyTorch is used
for device memory and streams only; every operator runs in the CUDA library.

Vectors are contiguous torch tensors in the library layout
[comp][elem][z][y][x]: float64 for the FP64 operators, float32 for the
multigrid-level entry points.  CUDA tensors are used in place on the
context's stream; CPU tensors are staged by the library (the call then blocks
until the result is back on the host).
"""
import ctypes

import torch

from . import _lib
from ._lib import SPACE_P, SPACE_U, check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One DG discretisation on a periodic Cartesian mesh (one GPU)."""

    def __init__(self, n_elem, degree, degree_p=-1, lo=(-torch.pi,) * 3, hi=(torch.pi,) * 3,
                 n_q_conv=0, penalty_factor=1.0, nu=1.0 / 1600, mg_coarse_n=2, mg_precision=32,
                 fp64_mode=0, stream=None):
        self.lib = _lib.load()
        if isinstance(n_elem, int):
            n_elem = (n_elem,) * 3
        d = _lib.MeshDesc()
        self.lib.dgns_default_desc(ctypes.byref(d))
        for i in range(3):
            d.n_elem[i] = int(n_elem[i])
            d.lo[i] = float(lo[i])
            d.hi[i] = float(hi[i])
        d.degree = int(degree)
        d.degree_p = int(degree_p)
        d.n_q_conv = int(n_q_conv)
        d.penalty_factor = float(penalty_factor)
        d.nu = float(nu)
        d.mg_coarse_n = int(mg_coarse_n)
        d.mg_precision = int(mg_precision)
        d.fp64_mode = int(fp64_mode)
        self.desc = d
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        h = ctypes.c_void_p()
        check(self.lib.dgns_create(ctypes.byref(d), sp, ctypes.byref(h)))
        self.h = h
        nu_, np_ = ctypes.c_longlong(), ctypes.c_longlong()
        check(self.lib.dgns_sizes(h, ctypes.byref(nu_), ctypes.byref(np_)))
        self.n_u, self.n_p = nu_.value, np_.value
        self.n_elem = tuple(int(v) for v in n_elem)
        self.degree = int(degree)
        self.degree_p = int(degree_p) if degree_p >= 0 else int(degree) - 1

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def size(self, space):
        return self.n_u if space == SPACE_U else self.n_p

    def nodes_1d(self, space=SPACE_U):
        n = (self.degree if space == SPACE_U else self.degree_p) + 1
        out = (ctypes.c_double * n)()
        check(self.lib.dgns_nodes_1d(self.h, space, out))
        return list(out)

    def _vec(self, t, numel, dtype=torch.float64, name="vector"):
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch.Tensor" % name)
        if t.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() != numel:
            raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), numel))
        return _ptr(t)

    def set_stream(self, stream):
        self.stream = stream
        check(self.lib.dgns_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    # ---------------------------------------------------------- operators
    def vmult_laplace(self, dst, src, space=SPACE_P):
        n = self.size(space)
        check(self.lib.dgns_vmult_laplace(self.h, self._vec(dst, n, name="dst"),
                                          self._vec(src, n, name="src"), space))
        return dst

    def vmult_laplace_split(self, dst, src, space=SPACE_P):
        """The SIPG Laplacian as separate cell, face and face-apply kernels
        (native FP64), for comparison with vmult_laplace."""
        n = self.size(space)
        check(self.lib.dgns_vmult_laplace_split(self.h, self._vec(dst, n, name="dst"),
                                                self._vec(src, n, name="src"), space))
        return dst

    def vmult_laplace_f32(self, dst, src, level):
        n = src.numel()
        check(self.lib.dgns_vmult_laplace_f32(self.h, self._vec(dst, n, torch.float32, "dst"),
                                              self._vec(src, n, torch.float32, "src"), level))
        return dst

    def laplace_diagonal(self, dst, space=SPACE_P):
        check(self.lib.dgns_laplace_diagonal(self.h, self._vec(dst, self.size(space), name="dst"), space))
        return dst

    def vmult_viscous(self, dst3, src3):
        n = 3 * self.n_u
        check(self.lib.dgns_vmult_viscous(self.h, self._vec(dst3, n, name="dst3"),
                                          self._vec(src3, n, name="src3")))
        return dst3

    def vmult_helmholtz(self, dst3, src3, mass_factor):
        n = 3 * self.n_u
        check(self.lib.dgns_vmult_helmholtz(self.h, self._vec(dst3, n, name="dst3"),
                                            self._vec(src3, n, name="src3"), float(mass_factor)))
        return dst3

    def vmult_mass(self, dst, src, ncomp=1, space=SPACE_U):
        n = ncomp * self.size(space)
        check(self.lib.dgns_vmult_mass(self.h, self._vec(dst, n, name="dst"),
                                       self._vec(src, n, name="src"), ncomp, space))
        return dst

    def apply_inverse_mass(self, dst, src, ncomp=1, space=SPACE_U):
        n = ncomp * self.size(space)
        check(self.lib.dgns_apply_inverse_mass(self.h, self._vec(dst, n, name="dst"),
                                               self._vec(src, n, name="src"), ncomp, space))
        return dst

    def vmult_divergence(self, dst_p, u3):
        check(self.lib.dgns_vmult_divergence(self.h, self._vec(dst_p, self.n_p, name="dst_p"),
                                             self._vec(u3, 3 * self.n_u, name="u3")))
        return dst_p

    def vmult_gradient(self, dst3, p):
        check(self.lib.dgns_vmult_gradient(self.h, self._vec(dst3, 3 * self.n_u, name="dst3"),
                                           self._vec(p, self.n_p, name="p")))
        return dst3

    def vmult_convective(self, dst3, u3):
        n = 3 * self.n_u
        check(self.lib.dgns_vmult_convective(self.h, self._vec(dst3, n, name="dst3"),
                                             self._vec(u3, n, name="u3")))
        return dst3

    def convective_face_size(self):
        n = ctypes.c_longlong()
        check(self.lib.dgns_convective_face_size(self.h, ctypes.byref(n)))
        return n.value

    def convective_faces(self, rface, u3):
        check(self.lib.dgns_convective_faces(self.h, self._vec(rface, self.convective_face_size(), name="rface"),
                                             self._vec(u3, 3 * self.n_u, name="u3")))
        return rface

    def convective_cells(self, dst3, u3, rface):
        n = 3 * self.n_u
        check(self.lib.dgns_convective_cells(self.h, self._vec(dst3, n, name="dst3"), self._vec(u3, n, name="u3"),
                                             self._vec(rface, self.convective_face_size(), name="rface")))
        return dst3

    def vjp_convective(self, grad_u3, u3, w3):
        n = 3 * self.n_u
        check(self.lib.dgns_vjp_convective(self.h, self._vec(grad_u3, n, name="grad_u3"),
                                           self._vec(u3, n, name="u3"), self._vec(w3, n, name="w3")))
        return grad_u3

    def dissipation(self, u3):
        out = ctypes.c_double()
        check(self.lib.dgns_dissipation(self.h, self._vec(u3, 3 * self.n_u, name="u3"), ctypes.byref(out)))
        return out.value

    def dissipation_grad(self, grad3, u3):
        n = 3 * self.n_u
        check(self.lib.dgns_dissipation_grad(self.h, self._vec(grad3, n, name="grad3"),
                                             self._vec(u3, n, name="u3")))
        return grad3

    def axpby(self, y, x, a, b):
        """y = a x + b y (device tensors of equal size)."""
        n = y.numel()
        check(self.lib.dgns_axpby(self.h, self._vec(y, n, name="y"), self._vec(x, n, name="x"),
                                  n, float(a), float(b)))
        return y

    def dot(self, a, b):
        out = ctypes.c_double()
        n = a.numel()
        check(self.lib.dgns_dot(self.h, self._vec(a, n, name="a"), self._vec(b, n, name="b"), n,
                                ctypes.byref(out)))
        return out.value

    def penalty_parameters(self, u_ex3, dt, zeta_d=1.0, zeta_c=1.0):
        """Per-cell (tau_D, tau_C) of the projection step, device tensors."""
        E = self.n_u // (self.degree + 1) ** 3
        td = torch.empty(E, dtype=torch.float64, device=u_ex3.device)
        tc = torch.empty_like(td)
        check(self.lib.dgns_penalty_parameters(self.h, self._vec(u_ex3, 3 * self.n_u, name="u_ex3"),
                                               float(dt), float(zeta_d), float(zeta_c), _ptr(td), _ptr(tc)))
        return td, tc

    def vmult_projection(self, dst3, src3, tau_d, tau_c, terms=_lib.PROJ_ALL):
        """dst3 = (M + A_D + A_C) src3 in one fused kernel, or one term of it
        (terms = PROJ_MASS, PROJ_DIV, PROJ_CONT) in its own pass."""
        n = 3 * self.n_u
        if terms == _lib.PROJ_ALL:
            check(self.lib.dgns_vmult_projection(self.h, self._vec(dst3, n, name="dst3"),
                                                 self._vec(src3, n, name="src3"), _ptr(tau_d), _ptr(tau_c)))
        else:
            td = _ptr(tau_d) if tau_d is not None else None
            tc = _ptr(tau_c) if tau_c is not None else None
            check(self.lib.dgns_vmult_projection_terms(self.h, self._vec(dst3, n, name="dst3"),
                                                       self._vec(src3, n, name="src3"), td, tc, int(terms)))
        return dst3

    # ------------------------------------------------------------ solvers
    @staticmethod
    def solve_params(**kw):
        p = _lib.SolveParams()
        _lib.load().dgns_default_solve_params(ctypes.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        return p

    @staticmethod
    def _info(info):
        return {k: getattr(info, k) for k, _ in _lib.SolveInfo._fields_}

    def cg_mg_solve(self, x, b, raise_on_error=True, **kw):
        p = self.solve_params(**kw)
        info = _lib.SolveInfo()
        rc = self.lib.dgns_cg_mg_solve(self.h, self._vec(x, self.n_p, name="x"),
                                       self._vec(b, self.n_p, name="b"), ctypes.byref(p),
                                       ctypes.byref(info))
        if raise_on_error:
            check(rc)
        out = self._info(info)
        out["rc"] = rc
        return out

    def cg_invmass_solve(self, x3, b3, mass_factor, raise_on_error=True, **kw):
        p = self.solve_params(**kw)
        info = _lib.SolveInfo()
        n = 3 * self.n_u
        rc = self.lib.dgns_cg_invmass_solve(self.h, self._vec(x3, n, name="x3"),
                                            self._vec(b3, n, name="b3"), float(mass_factor),
                                            ctypes.byref(p), ctypes.byref(info))
        if raise_on_error:
            check(rc)
        out = self._info(info)
        out["rc"] = rc
        return out

    def cg_projection_solve(self, x3, b3, tau_d, tau_c, raise_on_error=True, **kw):
        p = self.solve_params(**kw)
        info = _lib.SolveInfo()
        n = 3 * self.n_u
        rc = self.lib.dgns_cg_projection_solve(self.h, self._vec(x3, n, name="x3"), self._vec(b3, n, name="b3"),
                                               _ptr(tau_d), _ptr(tau_c), ctypes.byref(p), ctypes.byref(info))
        if raise_on_error:
            check(rc)
        out = self._info(info)
        out["rc"] = rc
        return out

    def mg_info(self):
        nl = ctypes.c_int()
        ne = (ctypes.c_int * _lib.MAX_LEVELS)()
        lam = (ctypes.c_double * _lib.MAX_LEVELS)()
        check(self.lib.dgns_mg_info(self.h, ctypes.byref(nl), ne, lam))
        return {"levels": nl.value, "n_elem": list(ne)[:nl.value], "lambda_max": list(lam)[:nl.value]}

    def mg_vcycle(self, z, r, **kw):
        p = self.solve_params(**kw)
        check(self.lib.dgns_mg_vcycle(self.h, self._vec(z, self.n_p, name="z"),
                                      self._vec(r, self.n_p, name="r"), ctypes.byref(p)))
        return z

    def mg_chebyshev_step_f32(self, dst, x, xprev, b, c1, c2, level):
        """dst = x + c1 (x - xprev) + c2 D^-1 (b - L x) on a multigrid level
        (FP32 device tensors; xprev None reads as zero)."""
        n = x.numel()
        xp = self._vec(xprev, n, torch.float32, "xprev") if xprev is not None else None
        check(self.lib.dgns_mg_chebyshev_step_f32(self.h, self._vec(dst, n, torch.float32, "dst"),
                                                  self._vec(x, n, torch.float32, "x"), xp,
                                                  self._vec(b, n, torch.float32, "b"), float(c1), float(c2),
                                                  int(level)))
        return dst

    def mg_prolongate_f32(self, fine, coarse, level):
        check(self.lib.dgns_mg_prolongate_f32(self.h, _ptr(fine), _ptr(coarse), level))
        return fine

    def mg_restrict_f32(self, coarse, fine, level):
        check(self.lib.dgns_mg_restrict_f32(self.h, _ptr(coarse), _ptr(fine), level))
        return coarse
