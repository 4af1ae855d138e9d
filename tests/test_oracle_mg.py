"""Pins of the oracle's multigrid and solver components (no GPU).

  transfers   prolongation reproduces polynomials exactly (it is an embedding);
              restriction is its transpose; P^T M_fine P = M_coarse (Galerkin
              identity of nested spaces)
  Chebyshev   on a diagonal matrix the error follows the closed form
              T_m((theta - lambda)/delta) / T_m(theta/delta)
  PCG         matches a dense solve; with the V-cycle as preconditioner the
              periodic Poisson problem converges in a mesh-independent number
              of iterations (Sec. 3.3 and Table of iteration counts, Sec. 4.3)
  V-cycle     column by column equal to the closed form built from dense level
              matrices, P, R = P^T and the Chebyshev polynomials evaluated on
              the eigen-decomposition (two and three levels); symmetric;
              a restriction scaled as an average, a dropped post-smoothing, a
              wrong coarse interval or degree each fail the closed form
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


# ---------------------------------------------------------------- V-cycle pins
# The V-cycle is a composition (pre-smoothing from a zero guess, residual,
# restriction, coarse correction, prolongation, post-smoothing).  Its pins
# below do not re-run the oracle's recursion: they build the operator from
# dense level matrices and the closed form of the Chebyshev polynomial, and
# check the oracle against it; planted mistakes of the composition fail them.

def _cheb_matrix(A, inv_diag, lam_max, rng, m):
    """Dense S with x = S b for m Jacobi-Chebyshev updates from a zero guess
    on [lam_max/rng, lam_max]: S = q(D^-1 A) D^-1 with q(t) = (1 - r_m(t))/t,
    r_m(t) = T_m((theta - t)/delta) / T_m(theta/delta) the residual polynomial
    (Saad, Sec. 12.1).  Evaluated on the eigen-decomposition of the
    symmetric D^-1/2 A D^-1/2; q(0) = -r_m'(0) for the null space."""
    lmin = lam_max / rng
    theta, delta = 0.5 * (lam_max + lmin), 0.5 * (lam_max - lmin)
    Tm = np.polynomial.chebyshev.Chebyshev.basis(m)
    s = np.sqrt(inv_diag)
    lam, U = np.linalg.eigh(s[:, None] * A * s[None, :])
    r = Tm((theta - lam) / delta) / Tm(theta / delta)
    dr0 = -Tm.deriv()(theta / delta) / delta / Tm(theta / delta)      # r_m'(0)
    small = np.abs(lam) < 1e-10 * lam.max()
    q = np.where(small, -dr0, (1.0 - r) / np.where(small, 1.0, lam))
    return s[:, None] * (U * q) @ U.T * s[None, :]


def _dense_levels(H):
    A = [lv["op"].matrix() for lv in H.levels]
    D = [lv["inv_diag"].ravel() for lv in H.levels]
    P = []
    for T in H.transfers:                     # P[:, j] = embedding of coarse unit vector j
        nc = T.cs.size
        cols = []
        for j in range(nc):
            e = np.zeros(nc)
            e[j] = 1.0
            cols.append(T.prolongate(e.reshape(T.cs.mesh.E, -1)).ravel())
        P.append(np.stack(cols, axis=1))
    return A, D, P


def _closed_form_vcycle(A, D, P, lam, degree, rng, coarse_iters):
    """B_0 = coarse Chebyshev (coarse_iters updates); on finer levels
    B_l = 2S - S A S + (I - S A) P B_{l-1} P^T (I - A S), the operator of
    pre-smoothing from zero, coarse correction with restriction P^T, and
    post-smoothing from the corrected iterate with the same polynomial."""
    B = _cheb_matrix(A[0], D[0], lam[0], rng, coarse_iters)
    for l in range(1, len(A)):
        S = _cheb_matrix(A[l], D[l], lam[l], rng, degree)
        I = np.eye(A[l].shape[0])
        B = 2 * S - S @ A[l] @ S + (I - S @ A[l]) @ P[l - 1] @ B @ P[l - 1].T @ (I - A[l] @ S)
    return B


def _oracle_vcycle_matrix(H, lam, degree, rng, coarse_iters):
    s = H.levels[-1]["space"]
    cols = []
    for j in range(s.size):
        e = np.zeros(s.size)
        e[j] = 1.0
        cols.append(H.vcycle(e.reshape(s.mesh.E, -1), lam, degree, rng, coarse_iters).ravel())
    return np.stack(cols, axis=1)


def _lam(H):
    return [1.2 * _lambda_max_dense(lv["op"], lv["inv_diag"], lv["space"].size) for lv in H.levels]


# 4^3 cells halved to 2^3 (two levels), or to 2^3 and 1^3 (three levels)
VC_CASES = [((4, 4, 4), 1, 2), ((4, 4, 4), 1, 1), ((4, 2, 2), 2, 1)]


@pytest.mark.parametrize("n,k,coarse_n", VC_CASES)
def test_vcycle_equals_closed_form(n, k, coarse_n):
    H = mg.Hierarchy(dg.Mesh(n), k, coarse_n=coarse_n)
    assert len(H.levels) == (2 if coarse_n == 2 else 3) or n == (4, 2, 2)
    lam = _lam(H)
    A, D, P = _dense_levels(H)
    B = _closed_form_vcycle(A, D, P, lam, 5, 20.0, 20)
    V = _oracle_vcycle_matrix(H, lam, 5, 20.0, 20)
    assert np.max(np.abs(V - B)) <= 1e-12 * np.max(np.abs(B))


@pytest.mark.parametrize("n,k,coarse_n", VC_CASES[:2])
def test_vcycle_is_symmetric(n, k, coarse_n):
    """<V r, s> = <r, V s>: the post-smoother is the adjoint of the
    pre-smoother and the restriction the transpose of the prolongation."""
    H = mg.Hierarchy(dg.Mesh(n), k, coarse_n=coarse_n)
    lam = _lam(H)
    E = H.levels[-1]["space"].mesh.E
    for seed in range(3):
        r, s = rand((E, 8), 40 + seed), rand((E, 8), 50 + seed)
        vr, vs = H.vcycle(r, lam, coarse_iters=20), H.vcycle(s, lam, coarse_iters=20)
        lhs, rhs = float(np.sum(vr * s)), float(np.sum(r * vs))
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(vr) * np.linalg.norm(s)


def _vcycle_error(H, lam):
    A, D, P = _dense_levels(H)
    B = _closed_form_vcycle(A, D, P, lam, 5, 20.0, 20)
    V = _oracle_vcycle_matrix(H, lam, 5, 20.0, 20)
    return np.max(np.abs(V - B)) / np.max(np.abs(B))


def test_vcycle_planted_mistakes_fail(monkeypatch):
    """Each plausible mistake of the composition, planted in the oracle on
    the CPU, moves its V-cycle far from the closed form (and the symmetry
    check catches the dropped post-smoothing on its own)."""
    H = mg.Hierarchy(dg.Mesh((4, 4, 4)), 1, coarse_n=2)
    lam = _lam(H)
    assert _vcycle_error(H, lam) <= 1e-12

    # (a) restriction scaled as an average over the 8 children
    T = H.transfers[0]
    orig = T.restrict
    monkeypatch.setattr(T, "restrict", lambda Xf: orig(Xf) / 8.0)
    assert _vcycle_error(H, lam) > 1e-3
    monkeypatch.setattr(T, "restrict", orig)

    # (b) post-smoothing dropped: Chebyshev with an initial guess returns it
    real = mg.chebyshev
    monkeypatch.setattr(mg, "chebyshev",
                        lambda A, d, b, x0, *a: x0.copy() if x0 is not None else real(A, d, b, x0, *a))
    assert _vcycle_error(H, lam) > 1e-3
    r, s = rand((64, 8), 1), rand((64, 8), 2)
    lhs = float(np.sum(H.vcycle(r, lam, coarse_iters=20) * s))
    rhs = float(np.sum(r * H.vcycle(s, lam, coarse_iters=20)))
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)
    monkeypatch.setattr(mg, "chebyshev", real)

    # (c) the coarse solve run on a wrong interval ([lam/5, lam] instead of
    # [lam/20, lam]); (d) the coarse solve run with the smoothing degree.
    # (Taking the interval of another level is no mistake here: on a uniform
    # periodic mesh D^-1 A has the same largest eigenvalue on every level.)
    for wrong in (lambda A, d, b, x0, lm, rg, m: real(A, d, b, x0, lm, 5.0 if m == 20 else rg, m),
                  lambda A, d, b, x0, lm, rg, m: real(A, d, b, x0, lm, rg, 5 if m == 20 else m)):
        monkeypatch.setattr(mg, "chebyshev", wrong)
        assert _vcycle_error(H, lam) > 1e-3
    monkeypatch.setattr(mg, "chebyshev", real)
