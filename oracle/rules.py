"""1D quadrature rules and the nodal Lagrange basis (oracle; test infrastructure).

Sec. 3.2 of the paper: shape functions are tensor products of 1D Lagrange
polynomials with Legendre-Gauss-Lobatto (LGL) support points, and all integrals
use Gaussian quadrature with enough points to be exact on affine cells.

Everything is on the reference interval [0, 1].
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def _extended(dtype):
    return np.dtype(dtype) != np.dtype(np.float64)


def legendre(n, x):
    """P_n(x) and P_n'(x) on [-1, 1] by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and
    P_n' = n (x P_n - P_{n-1}) / (x^2 - 1) (interior points), in the
    precision of x."""
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1, n * (x * p1 - p0) / (x * x - 1)


def gauss(n, dtype=np.float64):
    """n-point Gauss-Legendre rule on [0,1] (library routine, then mapped).
    In a wider dtype (np.longdouble) the library's roots are polished by
    Newton steps on P_n in that precision and the weights are
    2 / ((1 - x^2) P_n'(x)^2)."""
    x, w = npleg.leggauss(n)
    if _extended(dtype):
        x = np.asarray(x, dtype=dtype)
        for _ in range(3):
            p, dp = legendre(n, x)
            x = x - p / dp
        _, dp = legendre(n, x)
        w = 2 / ((1 - x * x) * dp * dp)
    return (x + 1) / 2, w / 2


def lgl_nodes(k, dtype=np.float64):
    """k+1 Legendre-Gauss-Lobatto points on [0,1]: the end points and the
    roots of P_k' (Sec. 3.2, 'Legendre-Gauss-Lobatto nodes as support points').
    Roots come from numpy's Legendre companion matrix and are polished by
    Newton steps on P_k' (with P_k'' = (2x P_k' - k(k+1) P_k) / (1 - x^2) from
    Legendre's equation in a wider dtype)."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    dP = npleg.Legendre.basis(k).deriv()
    ddP = dP.deriv()
    r = np.sort(dP.roots().real) if k > 1 else np.zeros(0)
    for _ in range(3):
        r = r - dP(r) / ddP(r)
    if _extended(dtype):
        r = np.asarray(r, dtype=dtype)
        for _ in range(3):
            p, dp = legendre(k, r)
            r = r - dp * (1 - r * r) / (2 * r * dp - k * (k + 1) * p)
    one = np.ones(1, dtype=dtype)
    x = np.concatenate([-one, np.asarray(r, dtype=dtype), one])
    return (x + 1) / 2


def lagrange(nodes, x, dtype=np.float64):
    """Values V[q, j] = phi_j(x_q) and derivatives D[q, j] = phi_j'(x_q) of the
    Lagrange polynomials through `nodes`, from the product formula
    phi_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    nodes = np.asarray(nodes, dtype=dtype)
    x = np.atleast_1d(np.asarray(x, dtype=dtype))
    n = len(nodes)
    V = np.ones((len(x), n), dtype=dtype)
    D = np.zeros((len(x), n), dtype=dtype)
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
