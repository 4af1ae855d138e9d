"""1D quadrature rules and the nodal Lagrange basis (oracle; test infrastructure).

Sec. 3.2 of the paper: shape functions are tensor products of 1D Lagrange
polynomials with Legendre-Gauss-Lobatto (LGL) support points, and all integrals
use Gaussian quadrature with enough points to be exact on affine cells.

Everything is on the reference interval [0, 1].
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(n):
    """n-point Gauss-Legendre rule on [0,1] (library routine, then mapped)."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def lgl_nodes(k):
    """k+1 Legendre-Gauss-Lobatto points on [0,1]: the end points and the
    roots of P_k' (Sec. 3.2, 'Legendre-Gauss-Lobatto nodes as support points').
    Roots come from numpy's Legendre companion matrix and are polished by
    Newton steps on P_k'."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    dP = npleg.Legendre.basis(k).deriv()
    ddP = dP.deriv()
    r = np.sort(dP.roots().real) if k > 1 else np.zeros(0)
    for _ in range(3):
        r = r - dP(r) / ddP(r)
    x = np.concatenate([[-1.0], r, [1.0]])
    return 0.5 * (x + 1.0)


def lagrange(nodes, x):
    """Values V[q, j] = phi_j(x_q) and derivatives D[q, j] = phi_j'(x_q) of the
    Lagrange polynomials through `nodes`, from the product formula
    phi_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    D = np.zeros((len(x), n))
    for j in range(n):
        others = [m for m in range(n) if m != j]
        den = np.prod([nodes[j] - nodes[m] for m in others])
        num = np.ones_like(x)
        for m in others:
            num = num * (x - nodes[m])
        V[:, j] = num / den
        # derivative of the product: sum over the dropped factor l
        dsum = np.zeros_like(x)
        for l in others:
            term = np.ones_like(x)
            for m in others:
                if m != l:
                    term = term * (x - nodes[m])
            dsum += term
        D[:, j] = dsum / den
    return V, D
