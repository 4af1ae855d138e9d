"""Pins of the oracle's multigrid and solver components (no GPU).

  transfers   prolongation reproduces polynomials exactly (it is an embedding);
              restriction is its transpose; P^T M_fine P = M_coarse (Galerkin
              identity of nested spaces)
  Chebyshev   on a diagonal matrix the error follows the closed form
              T_m((theta - lambda)/delta) / T_m(theta/delta)
  PCG         matches a dense solve; with the V-cycle as preconditioner the
              periodic Poisson problem converges in a mesh-independent number
              of iterations (Sec. 3.3 and Table of iteration counts, Sec. 4.3)
"""
import numpy as np
import pytest

from oracle import dg, mg, solvers


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, shape)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prolongation_reproduces_polynomials(k):
    mc, mf = dg.Mesh((2, 1, 2)), dg.Mesh((4, 2, 4))
    sc, sf = dg.Space(mc, k), dg.Space(mf, k)
    T = mg.Transfer(sc, sf)
    c = rand(4, k)
    p = lambda x, y, z: c[0] * x ** k + c[1] * y ** k * z + c[2] * x * y * z ** (k - 1) + c[3]
    assert np.max(np.abs(T.prolongate(sc.interpolate(p)) - sf.interpolate(p))) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_restriction_is_the_transpose_of_prolongation(k):
    """restrict is a separate scatter-add; <R f, c> = <f, P c> for random
    fine and coarse vectors (one child per direction of a coarse cell with
    one cell along y included)."""
    mc, mf = dg.Mesh((2, 1, 2)), dg.Mesh((4, 2, 4))
    sc, sf = dg.Space(mc, k), dg.Space(mf, k)
    T = mg.Transfer(sc, sf)
    f = rand((mf.E, sf.ndofs_cell), 21)
    c = rand((mc.E, sc.ndofs_cell), 22)
    lhs = float(np.sum(T.restrict(f) * c))
    rhs = float(np.sum(f * T.prolongate(c)))
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(f)) * np.max(np.abs(c))


@pytest.mark.parametrize("k", [1, 3])
def test_restriction_galerkin_mass(k):
    mc, mf = dg.Mesh((2, 2, 1)), dg.Mesh((4, 4, 2))
    sc, sf = dg.Space(mc, k), dg.Space(mf, k)
    T = mg.Transfer(sc, sf)
    x = rand((mc.E, sc.ndofs_cell), 5)
    lhs = T.restrict(dg.Mass(sf).apply(T.prolongate(x)))
    rhs = dg.Mass(sc).apply(x)
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))


@pytest.mark.parametrize("degree", [1, 2, 5, 8])
def test_chebyshev_closed_form(degree):
    lam = np.linspace(0.05, 2.0, 40)
    b = rand(40, degree)
    lam_max, rng = 2.0, 20.0
    x = mg.chebyshev(lambda v: lam * v, np.ones(40), b, None, lam_max, rng, degree)
    lmin = lam_max / rng
    theta, delta = 0.5 * (lam_max + lmin), 0.5 * (lam_max - lmin)
    Tm = np.polynomial.chebyshev.Chebyshev.basis(degree)
    resid_poly = Tm((theta - lam) / delta) / Tm(theta / delta)
    ref = (1.0 - resid_poly) / lam * b
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))
    # nonzero initial guess: the error contracts by the same polynomial
    x0 = rand(40, 99)
    x = mg.chebyshev(lambda v: lam * v, np.ones(40), b, x0, lam_max, rng, degree)
    xs = b / lam
    assert np.max(np.abs((x - xs) - resid_poly * (x0 - xs))) < 1e-12 * np.max(np.abs(xs))


def test_pcg_dense():
    A = rand((30, 30), 1)
    A = A @ A.T + 30 * np.eye(30)
    b = rand(30, 2)
    x, it, hist = solvers.pcg(lambda v: A @ v, b, precond=lambda r: r / np.diag(A),
                              rel_tol=1e-13)
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-10
    assert hist[-1] <= 1e-13


def _lambda_max_dense(op, inv_diag, size):
    A = op.matrix()
    d = np.sqrt(inv_diag.ravel())
    return np.linalg.eigvalsh(d[:, None] * A * d[None, :])[-1]


@pytest.mark.parametrize("n", [4, 8])
def test_vcycle_pcg_periodic_poisson(n):
    k = 2
    m = dg.Mesh(n)
    H = mg.Hierarchy(m, k, coarse_n=2)
    lam = []
    for lv in H.levels:
        if lv["space"].size <= 1800:
            lam.append(1.2 * _lambda_max_dense(lv["op"], lv["inv_diag"], lv["space"].size))
        else:   # power iteration on D^-1 A for the larger level
            v = rand(lv["space"].size, 3).reshape(lv["space"].mesh.E, -1)
            for _ in range(60):
                w = lv["inv_diag"] * lv["op"].apply(v)
                est = np.linalg.norm(w) / np.linalg.norm(v)
                v = w / np.linalg.norm(w)
            lam.append(1.2 * est)
    s = H.levels[-1]["space"]
    L = H.levels[-1]["op"]
    b = solvers.mean_free(rand((m.E, s.ndofs_cell), 11))
    x, it, hist = solvers.pcg(L.apply, b, precond=lambda r: H.vcycle(r, lam, coarse_iters=20),
                              rel_tol=1e-10, max_iter=60, project=True)
    assert hist[-1] <= 1e-10
    assert it <= 25
    assert solvers.relative_residual(L.apply, x, b) < 2e-10
