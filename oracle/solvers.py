"""Preconditioned conjugate gradients and residual checks (oracle; test
infrastructure).

Sec. 3.3 of the paper: the pressure Poisson, projection and Helmholtz systems
are symmetric positive (semi-)definite and are solved by preconditioned CG.
The oracle does not try to reproduce the device iteration; it checks returned
solutions through its own FP64 residual and, on small cases, against a dense
pseudo-inverse.
"""
import numpy as np


def mean_free(x):
    """Euclidean projection onto the complement of the constants (the null
    space of the periodic SIPG Laplacian)."""
    return x - x.mean()


def pcg(apply_A, b, precond=None, rel_tol=1e-10, max_iter=500, project=False):
    """Textbook preconditioned CG from a zero initial guess.  Returns
    (x, iterations, relative residual history)."""
    x = np.zeros_like(b)
    r = mean_free(b) if project else b.copy()
    z = precond(r) if precond else r.copy()
    if project:
        z = mean_free(z)
    p = z.copy()
    rz = float(np.vdot(r, z))
    nb = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(r)) / nb]
    it = 0
    while hist[-1] > rel_tol and it < max_iter:
        Ap = apply_A(p)
        alpha = rz / float(np.vdot(p, Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        z = precond(r) if precond else r.copy()
        if project:
            z = mean_free(z)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        hist.append(float(np.linalg.norm(r)) / nb)
    return x, it, hist


def relative_residual(apply_A, x, b):
    return float(np.linalg.norm(b - apply_A(x)) / np.linalg.norm(b))
