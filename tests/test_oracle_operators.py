"""Pins of the oracle's DG operators against closed forms and invariants (no GPU).

Each test ties an operator of Sec. 3.2 of the paper to a fact that the
mathematics fixes, chosen so that a dropped term, a wrong sign, a wrong index
or a transposed block fails at least one of them:
  mass          integrals of polynomials, exact inverse
  Laplace       symmetry, PSD with the constants as null space, consistency
                with -Laplacian on polynomials, closed-form energies of a
                piecewise-constant and a sawtooth field (penalty and both
                symmetric face terms), spectral convergence on sin(x)
  div / grad    D^T = -G, annihilation of constants, consistency on polynomials
  convective    conservation, constants, a two-cell LLF closed form,
                consistency on polynomials, Taylor-Green closed form
  diagnostics   kinetic energy 1/8 and dissipation 3 nu / 4 of Taylor-Green
"""
import numpy as np
import pytest

from oracle import dg, rules

PI = np.pi


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, shape)


def interior_cells(mesh):
    """Cells whose closure does not touch the periodic seam."""
    ok = np.ones(mesh.E, dtype=bool)
    for a in range(3):
        ok &= (mesh.ijk[a] > 0) & (mesh.ijk[a] < mesh.n[a] - 1)
    return np.nonzero(ok)[0]


def cell_moments(space, f, extra=4):
    """int_e phi_i f dx for every cell, by an independent tensor Gauss rule
    with N + extra points (f a callable of x, y, z)."""
    m = space.mesh
    g, w = rules.gauss(space.N + extra)
    V, _ = rules.lagrange(space.nodes, g)
    Phi = dg.tensor3(V, V, V)
    W = np.kron(w, np.kron(w, w)) * np.prod(m.h)
    Q = len(g)
    q = np.arange(Q ** 3)
    loc = [g[q % Q], g[(q // Q) % Q], g[q // (Q * Q)]]
    X = [m.lo[a] + (m.ijk[a][:, None] + loc[a][None, :]) * m.h[a] for a in range(3)]
    F = f(*X)
    return (F * W[None, :]) @ Phi


# --------------------------------------------------------------------- mass
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_mass_integrals(k):
    m = dg.Mesh((3, 2, 4))
    s = dg.Space(m, k)
    M = dg.Mass(s)
    one = np.ones((m.E, s.ndofs_cell))
    assert abs(np.sum(one * M.apply(one)) - (2 * PI) ** 3) < 1e-11
    if k >= 2:
        x2 = s.interpolate(lambda x, y, z: x * x)
        assert abs(np.sum(one * M.apply(x2)) - (2 * PI) ** 2 * 2 * PI ** 3 / 3) < 1e-10
        xy = s.interpolate(lambda x, y, z: x * y)
        assert abs(np.sum(xy * M.apply(xy)) - 2 * PI * (2 * PI ** 3 / 3) ** 2) < 1e-9
    x = rand((m.E, s.ndofs_cell), k)
    assert np.max(np.abs(M.apply_inverse(M.apply(x)) - x)) < 1e-12


# ------------------------------------------------------------------ Laplace
@pytest.mark.parametrize("n,k", [((2, 2, 2), 2), ((1, 2, 3), 3), ((4, 4, 4), 3), ((2, 2, 2), 5)])
def test_laplace_symmetric_psd_nullspace(n, k):
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    A = dg.Laplace(s).matrix()
    nrm = np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) <= 1e-13 * nrm
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert abs(ev[0]) < 1e-11 * ev[-1]
    assert ev[1] > 1e-6 * ev[-1]
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-12 * nrm


@pytest.mark.parametrize("k", [2, 3, 4])
def test_laplace_consistency_polynomial(k):
    m = dg.Mesh((4, 3, 4))
    s = dg.Space(m, k)
    L = dg.Laplace(s)
    c = rand(6, 10 + k)
    p = lambda x, y, z: (c[0] * x ** k + c[1] * x * y ** (k - 1) + c[2] * y * z
                         + c[3] * z ** k * x ** (k - 2) + c[4] * (x + y + z))
    # -Laplacian of p, written out
    def mlap(x, y, z):
        r = -(c[0] * k * (k - 1) * x ** (k - 2) + c[1] * x * (k - 1) * (k - 2) * y ** max(k - 3, 0)
              + c[3] * (k * (k - 1) * z ** (k - 2) * x ** (k - 2)
                        + z ** k * (k - 2) * (k - 3) * x ** max(k - 4, 0)))
        return r
    y = L.apply(s.interpolate(p))
    ref = cell_moments(s, mlap)
    cells = interior_cells(m)
    assert len(cells) > 0
    err = np.max(np.abs(y[cells] - ref[cells]))
    assert err < 1e-11 * max(1.0, np.max(np.abs(ref[cells])))


@pytest.mark.parametrize("k,pf", [(1, 1.0), (3, 1.0), (4, 2.5)])
def test_laplace_penalty_energy(k, pf):
    """Piecewise constant field: only tau [p]^2 survives."""
    m = dg.Mesh((3, 2, 4), lo=(-1.0, 0.0, -2.0), hi=(2.0, 1.0, 2.0))
    s = dg.Space(m, k)
    L = dg.Laplace(s, penalty_factor=pf)
    cval = rand(m.E, 3)
    P = np.repeat(cval[:, None], s.ndofs_cell, axis=1)
    energy = np.sum(P * L.apply(P))
    ref = 0.0
    for a in range(3):
        tau = pf * (k + 1) ** 2 / m.h[a]
        area = np.prod([m.h[b] for b in range(3) if b != a])
        ref += tau * area * np.sum((cval - cval[m.neighbor(a, +1)]) ** 2)
    assert abs(energy - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("k,axis", [(1, 0), (2, 1), (3, 2), (5, 0)])
def test_laplace_sawtooth_energy(k, axis):
    """p = distance from the cell's lower face along `axis`:
    energy = V - 2 sum_F h |F| + tau h^2 sum_F |F| over faces normal to axis."""
    m = dg.Mesh((2, 3, 2), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.5, 3.0))
    s = dg.Space(m, k)
    L = dg.Laplace(s)
    X = s.node_coords()[axis]
    P = X - (m.lo[axis] + m.ijk[axis][:, None] * m.h[axis])
    energy = np.sum(P * L.apply(P))
    h = m.h[axis]
    area = np.prod([m.h[b] for b in range(3) if b != axis])
    tau = (k + 1) ** 2 / h
    ref = m.volume + m.E * area * (-2.0 * h + tau * h * h)
    assert abs(energy - ref) < 1e-11 * abs(ref)


def test_laplace_spectral_convergence():
    """sin(x)cos(z) is an eigenfunction of -Laplacian with eigenvalue 2: the
    discrete Rayleigh quotient converges to it at a high rate, and pointwise
    M^-1 L u converges to 2u (at the lifted-jump rate h^(k-1))."""
    rq, errs = [], []
    for n in (2, 4):
        m = dg.Mesh(n)
        s = dg.Space(m, 3)
        u = s.interpolate(lambda x, y, z: np.sin(x) * np.cos(z))
        Lu = dg.Laplace(s).apply(u)
        rq.append(abs(np.sum(u * Lu) / np.sum(u * dg.Mass(s).apply(u)) - 2.0))
    assert rq[1] < rq[0] / 30.0 and rq[1] < 1e-3
    for n in (8, 16):
        m = dg.Mesh((n, 1, n))
        s = dg.Space(m, 3)
        u = s.interpolate(lambda x, y, z: np.sin(x) * np.cos(z))
        v = dg.Mass(s).apply_inverse(dg.Laplace(s).apply(u))
        errs.append(np.max(np.abs(v - 2.0 * u)))
    assert errs[1] < errs[0] / 3.0 and errs[1] < 0.02


def test_viscous_is_nu_laplace():
    m = dg.Mesh(2)
    s = dg.Space(m, 2)
    x = rand((m.E, s.ndofs_cell), 0)
    nu = 1.0 / 1600
    assert np.max(np.abs(dg.Viscous(s, nu).apply(x) - nu * dg.Laplace(s).apply(x))) < 1e-16


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 1, 3)])
def test_laplace_diagonal(n):
    m = dg.Mesh(n)
    s = dg.Space(m, 2)
    L = dg.Laplace(s)
    assert np.max(np.abs(L.diagonal().ravel() - np.diag(L.matrix()))) < 1e-12


# --------------------------------------------------------------- div / grad
@pytest.mark.parametrize("n,ku", [((2, 2, 2), 2), ((1, 2, 3), 3), ((3, 3, 2), 4)])
def test_divergence_gradient_adjoint(n, ku):
    m = dg.Mesh(n)
    su, sp = dg.Space(m, ku), dg.Space(m, ku - 1)
    D, G = dg.Divergence(su, sp), dg.Gradient(su, sp)
    nu_, np_ = su.size, sp.size
    Dm = np.stack([D.apply(e.reshape(3, m.E, -1)).ravel() for e in np.eye(3 * nu_)], 1)
    Gm = np.stack([G.apply(e.reshape(m.E, -1)).ravel() for e in np.eye(np_)], 1)
    assert np.max(np.abs(Dm.T + Gm)) < 1e-13 * np.max(np.abs(Dm))
    assert np.max(np.abs(Dm @ np.ones(3 * nu_))) < 1e-12 * np.max(np.abs(Dm))
    assert np.max(np.abs(Gm @ np.ones(np_))) < 1e-12 * np.max(np.abs(Gm))


@pytest.mark.parametrize("ku", [2, 3, 4])
def test_divergence_gradient_consistency(ku):
    m = dg.Mesh((4, 3, 3))
    su, sp = dg.Space(m, ku), dg.Space(m, ku - 1)
    c = rand(4, ku)
    ux = lambda x, y, z: c[0] * x ** ku + y * z
    uy = lambda x, y, z: c[1] * x * y ** (ku - 1) + z
    uz = lambda x, y, z: c[2] * z ** ku * y
    divu = lambda x, y, z: (c[0] * ku * x ** (ku - 1) + c[1] * (ku - 1) * x * y ** (ku - 2)
                            + c[2] * ku * z ** (ku - 1) * y)
    U = np.stack([su.interpolate(f) for f in (ux, uy, uz)])
    cells = interior_cells(m)
    y = dg.Divergence(su, sp).apply(U)
    ref = cell_moments(sp, divu)
    assert np.max(np.abs(y[cells] - ref[cells])) < 1e-11 * np.max(np.abs(ref[cells]))
    kp = ku - 1
    p = lambda x, y, z: c[3] * x ** kp * y + z ** kp + x * y * z
    grads = [lambda x, y, z: c[3] * kp * x ** (kp - 1) * y + y * z,
             lambda x, y, z: c[3] * x ** kp + x * z,
             lambda x, y, z: kp * z ** (kp - 1) + x * y]
    g = dg.Gradient(su, sp).apply(sp.interpolate(p))
    for a in range(3):
        ref = cell_moments(su, grads[a])
        assert np.max(np.abs(g[a][cells] - ref[cells])) < 1e-11 * np.max(np.abs(ref[cells]))


# --------------------------------------------------------------- convective
@pytest.mark.parametrize("n,k", [((2, 2, 2), 2), ((3, 1, 2), 3), ((2, 2, 2), 5)])
def test_convective_conservation_and_constants(n, k):
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    C = dg.Convective(s)
    U = rand((3, m.E, s.ndofs_cell), 7)
    Y = C.apply(U)
    scale = np.max(np.abs(Y))
    assert np.max(np.abs(Y.sum(axis=(1, 2)))) < 1e-12 * scale * Y[0].size
    const = np.stack([np.full((m.E, s.ndofs_cell), v) for v in (0.3, -1.2, 2.0)])
    assert np.max(np.abs(C.apply(const))) < 1e-12


def test_convective_two_cell_llf():
    """u = (a,0,0) on cell 0 and (b,0,0) on cell 1 of a 2x1x1 mesh: summing the
    x-component over the nodes of cell 0 leaves only the LLF jump terms,
    area * 2 max(|a|,|b|) (a - b)."""
    m = dg.Mesh((2, 1, 1), lo=(0, 0, 0), hi=(2.0, 1.0, 1.0))
    s = dg.Space(m, 2)
    a, b = 0.7, -1.3
    U = np.zeros((3, m.E, s.ndofs_cell))
    U[0][0], U[0][1] = a, b
    Y = dg.Convective(s).apply(U)
    area = m.h[1] * m.h[2]
    assert abs(Y[0][0].sum() - area * 2 * max(abs(a), abs(b)) * (a - b)) < 1e-13
    assert abs(Y[0][1].sum() + area * 2 * max(abs(a), abs(b)) * (a - b)) < 1e-13
    assert np.max(np.abs(Y[1:])) < 1e-14


@pytest.mark.parametrize("k", [2, 3])
def test_convective_consistency_polynomial(k):
    m = dg.Mesh((3, 3, 4))
    s = dg.Space(m, k)
    c = rand(3, 20 + k)
    f = [lambda x, y, z: c[0] * x ** k + y, lambda x, y, z: c[1] * y * x + z ** k,
         lambda x, y, z: c[2] * z * y ** (k - 1) + x]
    U = np.stack([s.interpolate(g) for g in f])
    Y = dg.Convective(s).apply(U)
    # div(u (x) u)_c = sum_d d_d (u_c u_d), by central differences of exact
    # polynomials is too crude; use the product rule with exact derivatives
    der = {
        (0, 0): lambda x, y, z: c[0] * k * x ** (k - 1), (0, 1): lambda x, y, z: 1.0 + 0 * x,
        (0, 2): lambda x, y, z: 0 * x, (1, 0): lambda x, y, z: c[1] * y,
        (1, 1): lambda x, y, z: c[1] * x, (1, 2): lambda x, y, z: k * z ** (k - 1),
        (2, 0): lambda x, y, z: 1.0 + 0 * x,
        (2, 1): lambda x, y, z: c[2] * z * (k - 1) * y ** (k - 2), (2, 2): lambda x, y, z: c[2] * y ** (k - 1)}
    cells = interior_cells(m)
    for comp in range(3):
        def rhs(x, y, z, comp=comp):
            u = [g(x, y, z) for g in f]
            divu = sum(der[(d, d)](x, y, z) for d in range(3))
            adv = sum(u[d] * der[(comp, d)](x, y, z) for d in range(3))
            return adv + u[comp] * divu
        ref = cell_moments(s, rhs, extra=k + 2)
        assert np.max(np.abs(Y[comp][cells] - ref[cells])) < 1e-11 * np.max(np.abs(ref[cells]))


def test_convective_taylor_green_closed_form():
    errs = []
    for n in (4, 8):
        m = dg.Mesh(n)
        s = dg.Space(m, 3)
        U = np.stack(s.interpolate(dg.taylor_green))
        V = dg.Mass(s).apply_inverse(dg.Convective(s).apply(U))
        X = s.node_coords()
        ref = np.stack([0.5 * np.sin(2 * X[0]) * np.cos(X[2]) ** 2,
                        0.5 * np.sin(2 * X[1]) * np.cos(X[2]) ** 2, 0 * X[0]])
        errs.append(np.max(np.abs(V - ref)))
    assert errs[1] < errs[0] / 6.0 and errs[1] < 0.02


# -------------------------------------------------------------- diagnostics
def test_taylor_green_energy_and_dissipation():
    nu = 1.0 / 1600
    m = dg.Mesh(8)
    s = dg.Space(m, 4)
    U = np.stack(s.interpolate(dg.taylor_green))
    assert abs(dg.kinetic_energy(s, U) - 0.125) < 1e-4
    assert abs(dg.dissipation_rate(s, U, nu) / nu - 0.75) < 1e-3


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 2)])
def test_energy_and_dissipation_exact_for_polynomials(n):
    """u = (x^2, xy, z) on [0, 1]^3 lies in the degree-2 space, and the
    (k+1)-point Gauss rule integrates |u|^2 and grad u : grad u exactly:
    e_k = (1/5 + 1/9 + 1/3) / 2 = 29/90 and eps = nu (4/3 + 1/3 + 1/3 + 1)
    = 3 nu on any mesh (the broken gradient of a smooth field is its
    gradient)."""
    nu = 0.01
    m = dg.Mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))
    s = dg.Space(m, 2)
    U = np.stack(s.interpolate(lambda x, y, z: (x * x, x * y, z)))
    assert abs(dg.kinetic_energy(s, U) - 29.0 / 90.0) < 1e-14
    assert abs(dg.dissipation_rate(s, U, nu) - 3.0 * nu) < 1e-15


@pytest.mark.parametrize("n,k,field", [((2, 2, 2), 2, "rand"), ((3, 1, 2), 3, "tgv"), ((1, 2, 1), 4, "rand")])
def test_convective_vjp_adjoint_identity(n, k, field):
    """<w, J v> = <J^T w, v>, with J v from central differences of C, which
    are exact for the quadratic cell term and for the LLF term away from its
    kinks (a small step crosses none for these seeded fields)."""
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    C = dg.Convective(s)
    if field == "tgv":
        U = np.stack(s.interpolate(dg.taylor_green)) + 1e-3 * rand((3, m.E, s.ndofs_cell), 1)
    else:
        U = rand((3, m.E, s.ndofs_cell), 2)
    V = rand(U.shape, 3)
    Wt = rand(U.shape, 4)
    # near-zero normal velocities of the Taylor-Green field put LLF kinks close
    # to the base point: a smaller step keeps the difference quotient exact
    eps = 1e-8 if field == "tgv" else 1e-6
    Jv = (C.apply(U + eps * V) - C.apply(U - eps * V)) / (2 * eps)
    lhs = np.sum(Wt * Jv)
    rhs = np.sum(C.vjp(U, Wt) * V)
    assert abs(lhs - rhs) < 1e-8 * np.sum(np.abs(Wt * Jv))


@pytest.mark.parametrize("n,k", [((1, 1, 1), 2), ((2, 1, 1), 1)])
def test_convective_vjp_against_the_full_jacobian(n, k):
    """J^T w elementwise: the Jacobian of C built column by column from
    central differences (a uniform offset keeps every normal velocity away
    from the LLF kinks, so each column is exact up to the difference error)."""
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    C = dg.Convective(s)
    U = rand((3, m.E, s.ndofs_cell), 31) * 0.2 + 0.7
    W = rand(U.shape, 32)
    eps = 1e-6
    J = np.empty((U.size, U.size))
    for j in range(U.size):
        e = np.zeros(U.size)
        e[j] = eps
        J[:, j] = ((C.apply(U + e.reshape(U.shape)) - C.apply(U - e.reshape(U.shape))) / (2 * eps)).ravel()
    ref = J.T @ W.ravel()
    assert np.max(np.abs(C.vjp(U, W).ravel() - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_convective_vjp_quadratic_exact():
    """Without kinks (u.n of one sign everywhere and |u-.n| > |u+.n| on all
    faces is not needed: use a field whose LLF lambda is constant), C is
    quadratic and C(u+v) - C(u-v) = 2 J(u) v exactly."""
    m = dg.Mesh((2, 2, 2))
    s = dg.Space(m, 2)
    C = dg.Convective(s)
    # constant (1, 1, 1) plus a tiny perturbation keeps lambda = |u.n| on the
    # side with the larger value; compare with a large step on the cell term
    U = np.ones((3, m.E, s.ndofs_cell)) * 3.0 + 0.1 * rand((3, m.E, s.ndofs_cell), 5)
    V = 0.1 * rand(U.shape, 6)
    Wt = rand(U.shape, 7)
    eps = 1e-3
    Jv = (C.apply(U + eps * V) - C.apply(U - eps * V)) / (2 * eps)
    assert abs(np.sum(Wt * Jv) - np.sum(C.vjp(U, Wt) * V)) < 1e-10 * np.sum(np.abs(Wt * Jv))


def test_dissipation_gradient_matches_difference_quotient():
    nu = 1.0 / 1600
    m = dg.Mesh((2, 3, 2))
    s = dg.Space(m, 3)
    U = rand((3, m.E, s.ndofs_cell), 8)
    V = rand(U.shape, 9)
    eps = 1e-3   # the functional is quadratic: the central difference is exact
    fd = (dg.dissipation_rate(s, U + eps * V, nu) - dg.dissipation_rate(s, U - eps * V, nu)) / (2 * eps)
    g = dg.dissipation_gradient(s, U, nu)
    assert abs(np.sum(g * V) - fd) < 1e-12 * abs(fd)
    assert abs(0.5 * np.sum(g * U) - dg.dissipation_rate(s, U, nu)) < 1e-13 * dg.dissipation_rate(s, U, nu)


# --------------------------------------------------------------- projection
def test_penalty_parameters_constant_field():
    m = dg.Mesh((3, 2, 2))
    s = dg.Space(m, 3)
    U = np.stack([np.full((m.E, s.ndofs_cell), v) for v in (1.0, 2.0, -2.0)])
    dt = 1e-3
    tau_d, tau_c = dg.penalty_parameters(s, U, dt, zeta_d=1.0, zeta_c=0.5)
    h = np.prod(m.h) ** (1 / 3)
    assert np.max(np.abs(tau_d - 3.0 * h / 4 * dt)) < 1e-15
    assert np.max(np.abs(tau_c - 1.5 * dt)) < 1e-15


def test_penalty_parameters_cellwise_average():
    """||u||_e is the volume average of |u| over each cell: for
    u = (1 + x, 0, 0) on [0, 3] x [0, 1] x [0, 2] with three cells along x
    (|u| is linear, so the (k+1)-point Gauss rule is exact), the averages are
    the values at the cell centres, 1.5, 2.5, 3.5, and h = (1 * 1 * 2)^(1/3)."""
    m = dg.Mesh((3, 1, 1), lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 2.0))
    k, dt = 2, 1e-2
    s = dg.Space(m, k)
    ux = np.stack(s.interpolate(lambda x, y, z: (1.0 + x, 0 * x, 0 * x)))
    tau_d, tau_c = dg.penalty_parameters(s, ux, dt, zeta_d=2.0, zeta_c=0.5)
    avg = np.array([1.5, 2.5, 3.5])
    h = 2.0 ** (1.0 / 3.0)
    assert np.max(np.abs(tau_d - 2.0 * avg * h / (k + 1) * dt)) < 1e-15
    assert np.max(np.abs(tau_c - 0.5 * avg * dt)) < 1e-15


@pytest.mark.parametrize("n,k", [((2, 2, 2), 2), ((1, 2, 3), 3)])
def test_projection_symmetric_and_mass_plus_psd(n, k):
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    rng = np.random.default_rng(4)
    P = dg.Projection(s, rng.uniform(0.1, 1.0, m.E), rng.uniform(0.1, 1.0, m.E))
    N3 = 3 * s.size
    A = np.stack([P.apply(e.reshape(3, m.E, -1)).ravel() for e in np.eye(N3)], 1)
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))
    Mb = np.kron(np.eye(3), np.kron(np.eye(m.E), dg.Mass(s).Me))
    assert np.linalg.eigvalsh(0.5 * (A + A.T) - Mb)[0] > -1e-12 * np.max(np.abs(A))


def test_projection_penalty_energies():
    """Sawtooth u_x = x - x_cell: div u = 1 in every cell, so u^T A_D u =
    sum tau_D V_e; its x-jumps are h: u^T A_C u = sum_faces {{tau_C}} |F| h^2.
    Piecewise constant u_y: no divergence, u^T A_C u = sum {{tau_C}} |F| [u_y]^2."""
    m = dg.Mesh((3, 2, 2), lo=(0, 0, 0), hi=(1.5, 1.0, 0.6))
    s = dg.Space(m, 3)
    rng = np.random.default_rng(5)
    td, tc = rng.uniform(0.1, 1.0, m.E), rng.uniform(0.1, 1.0, m.E)
    M = dg.Mass(s)
    X = s.node_coords()[0]
    U = np.zeros((3, m.E, s.ndofs_cell))
    U[0] = X - (m.lo[0] + m.ijk[0][:, None] * m.h[0])
    P = dg.Projection(s, td, tc)
    e = np.sum(U * P.apply(U)) - np.sum(U[0] * M.apply(U[0]))
    Ve = np.prod(m.h)
    ep = m.neighbor(0, +1)
    ref = np.sum(td) * Ve + np.sum(0.5 * (tc + tc[ep])) * m.h[1] * m.h[2] * m.h[0] ** 2
    assert abs(e - ref) < 1e-12 * ref
    cval = rng.uniform(-1, 1, m.E)
    U = np.zeros((3, m.E, s.ndofs_cell))
    U[1] = np.repeat(cval[:, None], s.ndofs_cell, 1)
    e = np.sum(U * P.apply(U)) - np.sum(U[1] * M.apply(U[1]))
    ey = m.neighbor(1, +1)
    ref = np.sum(0.5 * (tc + tc[ey]) * (cval - cval[ey]) ** 2) * m.h[0] * m.h[2]
    assert abs(e - ref) < 1e-12 * abs(ref)


def test_patch_centre_equals_full_mesh_output():
    """The basis of the full-size sampled parity tests: on the uniform periodic
    mesh every operator couples a cell only to its face neighbours and is
    translation invariant, so a cell's output equals the output of the centre
    cell of a 3x3x3 periodic patch (same cell size) holding it and its
    neighbours."""
    from paper_1802_01439_gb300 import inputs
    from tests.test_gpu_fullsize import CENTRE, _patch, _patch_space
    n, ku, kp = 4, 3, 2
    m = dg.Mesh(n)
    su, sp = dg.Space(m, ku), dg.Space(m, kp)
    psu, psp = _patch_space(n, ku), _patch_space(n, kp)
    U = inputs.uniform(3, 3 * su.size).reshape(3, m.E, -1)
    P = inputs.uniform(4, sp.size).reshape(1, m.E, -1)
    full = {"conv": dg.Convective(su).apply(U), "div": dg.Divergence(su, sp).apply(U)[None],
            "lap": dg.Laplace(sp).apply(P[0])[None], "grad": dg.Gradient(su, sp).apply(P[0]),
            "helm": dg.Helmholtz(su, 1 / 1600, 1500.0).apply(U[0])[None]}
    for e in (0, 21, m.E - 1):
        patch = {"conv": dg.Convective(psu).apply(_patch(U, n, e))[:, CENTRE],
                 "div": dg.Divergence(psu, psp).apply(_patch(U, n, e))[None, CENTRE],
                 "lap": dg.Laplace(psp).apply(_patch(P, n, e)[0])[None, CENTRE],
                 "grad": dg.Gradient(psu, psp).apply(_patch(P, n, e)[0])[:, CENTRE],
                 "helm": dg.Helmholtz(psu, 1 / 1600, 1500.0).apply(_patch(U, n, e)[0])[None, CENTRE]}
        for k in full:
            assert np.max(np.abs(full[k][:, e] - patch[k])) <= 1e-13 * np.max(np.abs(full[k])), (k, e)


def test_convective_magnitude_bounds_the_result():
    """magnitude(U) bounds |C(U)| elementwise (triangle inequality), is
    positive, scales quadratically, and exceeds |C(U)| clearly for a smooth
    field, whose weak-form sums cancel."""
    m = dg.Mesh((2, 3, 2))
    s = dg.Space(m, 3)
    C = dg.Convective(s)
    U = np.random.default_rng(5).uniform(-1, 1, (3, m.E, s.ndofs_cell))
    y, mag = C.apply(U), C.magnitude(U)
    assert np.all(np.abs(y) <= mag * (1 + 1e-12) + 1e-300)
    assert np.allclose(C.magnitude(2.0 * U), 4.0 * mag, rtol=1e-14, atol=0)
    assert np.all(mag > 0)
    # a smooth field: the weak form cancels, the magnitude does not
    ut = np.stack(s.interpolate(dg.taylor_green))
    assert np.max(np.abs(C.apply(ut))) < 0.5 * np.max(C.magnitude(ut))


def _brute_force_sipg(mesh, k, penalty_factor=1.0):
    """Global SIPG matrix entry by entry from the bilinear form (the cell
    terms of l_h of Sec. 3.2 and, per interior face with n = +e_a,
    -{{d_n q}} [p] - [q] {{d_n p}} + tau [q] [p], tau = pf (k+1)^2 / h_a),
    integrated by (k+2)-point Gauss quadrature in physical coordinates over
    every cell and face for every pair of global basis functions (tensor
    Lagrange polynomials on each cell's LGL nodes, zero outside it).  Shares
    nothing with the element and face matrices of dg.Laplace."""
    N, nq = k + 1, k + 2
    nodes = rules.lgl_nodes(k)
    xq, wq = rules.gauss(nq)
    V, D = rules.lagrange(nodes, xq)               # (nq, N) on [0, 1]
    V01, D01 = rules.lagrange(nodes, [0.0, 1.0])   # face values and derivatives
    h = mesh.h
    nd = N ** 3
    A = np.zeros((mesh.E * nd, mesh.E * nd))
    loc = [(i % N, (i // N) % N, i // (N * N)) for i in range(nd)]
    # cell terms: sum_d int (d_d phi_I)(d_d phi_J), d_d = (1/h_d) d/dxi_d
    grads = []
    for d in range(3):
        g = np.zeros((nq ** 3, nd))
        for i, (a, b, c) in enumerate(loc):
            f = [V[:, a], V[:, b], V[:, c]]
            f[d] = D[:, (a, b, c)[d]] / h[d]
            g[:, i] = np.kron(f[2], np.kron(f[1], f[0]))
        grads.append(g)
    w3 = np.kron(wq, np.kron(wq, wq)) * np.prod(h)
    Ke = sum(g.T @ (w3[:, None] * g) for g in grads)
    for e in range(mesh.E):
        A[e * nd:(e + 1) * nd, e * nd:(e + 1) * nd] += Ke
    # faces: e- = e (its layer xi_a = 1) and e+ = its +a neighbour (xi_a = 0)
    for a in range(3):
        t = [b for b in range(3) if b != a]
        wf = np.kron(wq, wq) * h[t[0]] * h[t[1]]
        tau = penalty_factor * (k + 1) ** 2 / h[a]
        nb = mesh.neighbor(a, +1)
        for e in range(mesh.E):
            jump = np.zeros((nq * nq, mesh.E * nd))
            avg = np.zeros((nq * nq, mesh.E * nd))
            for cell, side, sgn in ((e, 1, 1.0), (nb[e], 0, -1.0)):
                for i, ijk in enumerate(loc):
                    tang = np.kron(V[:, ijk[t[1]]], V[:, ijk[t[0]]])
                    val = V01[side, ijk[a]] * tang
                    dn = D01[side, ijk[a]] / h[a] * tang
                    jump[:, cell * nd + i] += sgn * val
                    avg[:, cell * nd + i] += 0.5 * dn
            A += (-avg.T @ (wf[:, None] * jump) - jump.T @ (wf[:, None] * avg)
                  + tau * jump.T @ (wf[:, None] * jump))
    return A


@pytest.mark.parametrize("n,k,lohi", [((1, 1, 1), 1, None), ((2, 1, 1), 2, None), ((2, 2, 1), 1, None),
                                      ((1, 2, 2), 3, ((0.0, -1.0, 0.5), (1.0, 2.0, 3.0))),
                                      ((3, 1, 1), 2, ((0.0, 0.0, 0.0), (1.5, 0.7, 2.0)))])
def test_laplace_matches_brute_force_assembly(n, k, lohi):
    """The oracle's element-and-face application equals the global matrix
    built pair by pair from the bilinear form (meshes with one cell per
    direction included: there a cell is its own periodic neighbour)."""
    m = dg.Mesh(n) if lohi is None else dg.Mesh(n, lo=lohi[0], hi=lohi[1])
    A = dg.Laplace(dg.Space(m, k)).matrix()
    B = _brute_force_sipg(m, k)
    assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))


def _lagrange_by_products(nodes, x):
    """Values and first derivatives of the Lagrange polynomials of `nodes` at
    the points x, written out as products (independent of rules.lagrange)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    val = np.zeros((len(x), n))
    der = np.zeros((len(x), n))
    for j in range(n):
        others = [nodes[m] for m in range(n) if m != j]
        den = np.prod([nodes[j] - xm for xm in others])
        val[:, j] = np.prod([x - xm for xm in others], axis=0) / den
        for l in range(len(others)):
            der[:, j] += np.prod([x - xm for m, xm in enumerate(others) if m != l], axis=0) / den
    return val, der


def _brute_force_convective(mesh, k, U):
    """c_h(u, phi_i) of Sec. 3.2 for every test function, by quadrature in
    physical coordinates cell by cell and face by face:
      cell:  -sum_d int u_c u_d d_d phi_i, by a (Q + 2)-point Gauss rule (the
             integrand is a polynomial of degree < 2Q + 3 per direction, so
             this is the exact integral);
      faces: for every cell e and axis a the face between e (its layer
             xi_a = 1) and the cell at integer offset +1 along a, n = +e_a,
             F*_c = {{u_c u_a}} + max(|u_a^-|, |u_a^+|)(u_c^- - u_c^+), tested
             with phi^- - phi^+; the central part again exactly (Q + 2
             points), the dissipative part with the Q-point Gauss rule of the
             3/2 over-integration, Q = floor(3(k+1)/2).
    U: (3, E, N^3) nodal values, x fastest.  Shares no table with
    dg.Convective: the basis is evaluated by products at the points of
    numpy's Gauss-Legendre rule."""
    N = k + 1
    Q = (3 * N) // 2
    nodes = np.asarray(rules.lgl_nodes(k))
    nx, ny, nz = mesh.n
    h = mesh.h

    def rule(n):
        x, w = np.polynomial.legendre.leggauss(n)
        return 0.5 * (x + 1.0), 0.5 * w

    def cell_of(i, j, l):
        return (i % nx) + nx * ((j % ny) + ny * (l % nz))

    def field(e, c):
        return U[c, e].reshape(N, N, N)            # [z, y, x]

    out = np.zeros_like(U)
    xe, we = rule(Q + 2)
    Ve, De = _lagrange_by_products(nodes, xe)
    jac = h[0] * h[1] * h[2]
    W3 = np.einsum("a,b,c->abc", we, we, we) * jac  # [pz, py, px]
    # cell terms
    for e in range(mesh.E):
        u = [np.einsum("zyx,az,by,cx->abc", field(e, c), Ve, Ve, Ve) for c in range(3)]
        for c in range(3):
            for d in range(3):
                f = u[c] * u[d] * W3
                B = [Ve, Ve, Ve]                   # per direction x, y, z
                B[d] = De / h[d]
                out[c, e] -= np.einsum("abc,az,by,cx->zyx", f, B[2], B[1], B[0]).ravel()
    # faces
    ends_v, _ = _lagrange_by_products(nodes, np.array([0.0, 1.0]))
    for a in range(3):
        t1, t2 = [b for b in range(3) if b != a]
        for part, (xf, wf) in (("central", rule(Q + 2)), ("llf", rule(Q))):
            Vf, _ = _lagrange_by_products(nodes, xf)
            Wf = np.outer(wf, wf) * h[t1] * h[t2]  # [p2, p1]

            def trace(e, c, layer):
                # the cell's field on its face layer xi_a = layer at the points (p2 along t2, p1 along t1)
                T = np.moveaxis(field(e, c), [2 - a, 2 - t1, 2 - t2], [0, 1, 2])   # [a, t1, t2]
                return np.einsum("ijk,i,pj,qk->qp", T, ends_v[layer], Vf, Vf)

            def test_with(e, c, layer, g):
                # add sum over points of g (shape [p2, p1]) times phi_i on the face layer to out[c, e]
                R = np.einsum("qp,i,pj,qk->ijk", g, ends_v[layer], Vf, Vf)       # [a, t1, t2]
                out[c, e] += np.moveaxis(R, [0, 1, 2], [2 - a, 2 - t1, 2 - t2]).ravel()

            for e in range(mesh.E):
                ijk = [int(v) for v in mesh.ijk[:, e]]
                ijk[a] += 1
                ep = cell_of(*ijk)
                um = [trace(e, c, 1) for c in range(3)]
                up = [trace(ep, c, 0) for c in range(3)]
                lam = np.maximum(np.abs(um[a]), np.abs(up[a]))
                for c in range(3):
                    if part == "central":
                        F = 0.5 * (um[c] * um[a] + up[c] * up[a])
                    else:
                        F = lam * (um[c] - up[c])
                    test_with(e, c, 1, F * Wf)
                    test_with(ep, c, 0, -F * Wf)
    return out


@pytest.mark.parametrize("n,k,lohi,field", [((1, 1, 1), 1, None, "rand"), ((2, 1, 1), 2, None, "rand"),
                                            ((2, 2, 1), 1, None, "tgv"),
                                            ((1, 2, 2), 3, ((0.0, -1.0, 0.5), (1.0, 2.0, 3.0)), "rand"),
                                            ((3, 1, 2), 2, ((0.0, 0.0, 0.0), (1.5, 0.7, 2.0)), "rand")])
def test_convective_matches_brute_force_quadrature(n, k, lohi, field):
    """The oracle's table-based C(U) equals the weak form integrated point by
    point in physical coordinates (exact integrals for the polynomial parts,
    the 3/2 rule for the Lax-Friedrichs part), on meshes with one cell per
    direction (a cell is its own periodic neighbour) and non-cubic cells."""
    m = dg.Mesh(n) if lohi is None else dg.Mesh(n, lo=lohi[0], hi=lohi[1])
    s = dg.Space(m, k)
    if field == "tgv":
        U = np.stack(s.interpolate(dg.taylor_green)) + 1e-3 * rand((3, m.E, s.ndofs_cell), 1)
    else:
        U = rand((3, m.E, s.ndofs_cell), 7)
    A = dg.Convective(s).apply(U)
    B = _brute_force_convective(m, k, U)
    assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))


def _face_basis(V, ends, layer, a):
    """[face point, node] table of a cell's basis on its layer xi_a = layer:
    V holds the N 1D functions at the face rule's points (the points of the
    two tangential directions t1 < t2, t1 fastest), ends their values at
    xi = 0 and 1."""
    N = V.shape[1]
    t1, t2 = [b for b in range(3) if b != a]
    out = np.zeros((V.shape[0] ** 2, N ** 3))
    for i in range(N ** 3):
        idx = (i % N, (i // N) % N, i // (N * N))
        out[:, i] = ends[layer, idx[a]] * np.kron(V[:, idx[t2]], V[:, idx[t1]])
    return out


def _brute_force_divergence(mesh, ku, kp):
    """Global matrix of d_h(q, u) of Sec. 3.2, rows the pressure basis
    functions, columns the velocity basis functions (component, cell, node):
      -int grad(q) . u over every cell
      + over every face between a cell e (its layer xi_a = 1) and the cell at
        integer offset +1 along a: int [q] {{u_a}}, [q] = q^- - q^+,
    with every integral taken exactly (a (k_u + 3)-point Gauss rule per
    direction, physical coordinates).  Basis functions by products on each
    cell's LGL nodes, zero outside it; shares no table with dg.Divergence."""
    Nu, Np = ku + 1, kp + 1
    nu3, np3 = Nu ** 3, Np ** 3
    x, w = np.polynomial.legendre.leggauss(ku + 3)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    Vu, Du = _lagrange_by_products(np.asarray(rules.lgl_nodes(ku)), x)
    Vp, Dp = _lagrange_by_products(np.asarray(rules.lgl_nodes(kp)), x)
    eu, _ = _lagrange_by_products(np.asarray(rules.lgl_nodes(ku)), np.array([0.0, 1.0]))
    ep_, _ = _lagrange_by_products(np.asarray(rules.lgl_nodes(kp)), np.array([0.0, 1.0]))
    h = mesh.h
    nx, ny, nz = mesh.n
    E = mesh.E
    B = np.zeros((E * np3, 3 * E * nu3))

    def tab3(T):
        # T = (tx, ty, tz) 1D tables over the same point set -> [point, node], x fastest in both
        return np.kron(T[2], np.kron(T[1], T[0]))

    wq = np.kron(w, np.kron(w, w)) * h[0] * h[1] * h[2]
    phi = tab3((Vu, Vu, Vu))
    for a in range(3):
        T = [Vp, Vp, Vp]
        T[a] = Dp / h[a]
        block = -(tab3(T).T @ (wq[:, None] * phi))
        for e in range(E):
            B[e * np3:(e + 1) * np3, (a * E + e) * nu3:(a * E + e + 1) * nu3] += block
    for a in range(3):
        t1, t2 = [b for b in range(3) if b != a]
        wf = np.kron(w, w) * h[t1] * h[t2]         # face points: t1 fastest

        qm, qp = _face_basis(Vp, ep_, 1, a), _face_basis(Vp, ep_, 0, a)
        um, up = _face_basis(Vu, eu, 1, a), _face_basis(Vu, eu, 0, a)
        for e in range(E):
            ijk = [int(v) for v in mesh.ijk[:, e]]
            ijk[a] += 1
            f = (ijk[0] % nx) + nx * ((ijk[1] % ny) + ny * (ijk[2] % nz))
            for row_cell, q, sq in ((e, qm, 1.0), (f, qp, -1.0)):
                for col_cell, u in ((e, um), (f, up)):
                    B[row_cell * np3:(row_cell + 1) * np3,
                      (a * E + col_cell) * nu3:(a * E + col_cell + 1) * nu3] += \
                        sq * 0.5 * (q.T @ (wf[:, None] * u))
    return B


@pytest.mark.parametrize("n,ku,kp,lohi", [((1, 1, 1), 2, 1, None), ((2, 1, 1), 3, 2, None),
                                          ((2, 2, 1), 1, 1, None),
                                          ((1, 2, 2), 2, 1, ((0.0, -1.0, 0.5), (1.0, 2.0, 3.0))),
                                          ((3, 1, 2), 3, 2, ((0.0, 0.0, 0.0), (1.5, 0.7, 2.0)))])
def test_divergence_gradient_match_brute_force_assembly(n, ku, kp, lohi):
    """The oracle's D equals the global matrix of d_h built pair by pair, and
    its G equals minus that matrix's transpose (meshes with one cell per
    direction and non-cubic cells included)."""
    m = dg.Mesh(n) if lohi is None else dg.Mesh(n, lo=lohi[0], hi=lohi[1])
    su, sp = dg.Space(m, ku), dg.Space(m, kp)
    B = _brute_force_divergence(m, ku, kp)
    U = rand((3, m.E, su.ndofs_cell), 11)
    P = rand((m.E, sp.ndofs_cell), 12)
    y = B @ U.ravel()
    g = -(B.T @ P.ravel())
    assert np.max(np.abs(dg.Divergence(su, sp).apply(U).ravel() - y)) <= 1e-12 * np.max(np.abs(y))
    assert np.max(np.abs(dg.Gradient(su, sp).apply(P).ravel() - g)) <= 1e-12 * np.max(np.abs(g))


def _brute_force_projection(mesh, k, tau_d, tau_c):
    """Global matrix of the projection operator M + A_D + A_C (Sec. 3.2 and
    3.3), pair by pair of global basis functions phi e_c (component, cell,
    node), every integral exact ((k + 3)-point Gauss rule, physical
    coordinates):
      mass:        int phi_I phi_J (same component);
      divergence:  tau_D(e) int_e d_b phi_I d_a phi_J (row component b,
                   column component a);
      continuity:  over every face between a cell e (layer xi_a = 1) and the
                   cell at integer offset +1 along a, with n = e_a:
                   {{tau_C}} int [v . n] [u . n], [w] = w^- - w^+ (component a
                   only)."""
    N = k + 1
    n3, E = N ** 3, mesh.E
    x, w = np.polynomial.legendre.leggauss(k + 3)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    nodes = np.asarray(rules.lgl_nodes(k))
    V, D = _lagrange_by_products(nodes, x)
    ends, _ = _lagrange_by_products(nodes, np.array([0.0, 1.0]))
    h = mesh.h
    nx, ny, nz = mesh.n
    A = np.zeros((3 * E * n3, 3 * E * n3))

    def blk(c, e):
        return slice((c * E + e) * n3, (c * E + e + 1) * n3)

    def tab3(T):
        return np.kron(T[2], np.kron(T[1], T[0]))

    wq = np.kron(w, np.kron(w, w)) * h[0] * h[1] * h[2]
    phi = tab3((V, V, V))
    dphi = []
    for a in range(3):
        T = [V, V, V]
        T[a] = D / h[a]
        dphi.append(tab3(T))
    Mloc = phi.T @ (wq[:, None] * phi)
    for e in range(E):
        for c in range(3):
            A[blk(c, e), blk(c, e)] += Mloc
        for b in range(3):
            for a in range(3):
                A[blk(b, e), blk(a, e)] += tau_d[e] * (dphi[b].T @ (wq[:, None] * dphi[a]))
    for a in range(3):
        t1, t2 = [b for b in range(3) if b != a]
        wf = np.kron(w, w) * h[t1] * h[t2]
        vm, vp = _face_basis(V, ends, 1, a), _face_basis(V, ends, 0, a)
        for e in range(E):
            ijk = [int(v) for v in mesh.ijk[:, e]]
            ijk[a] += 1
            f = (ijk[0] % nx) + nx * ((ijk[1] % ny) + ny * (ijk[2] % nz))
            tc = 0.5 * (tau_c[e] + tau_c[f])
            for ci, ti, si in ((e, vm, 1.0), (f, vp, -1.0)):
                for cj, tj, sj in ((e, vm, 1.0), (f, vp, -1.0)):
                    A[blk(a, ci), blk(a, cj)] += tc * si * sj * (ti.T @ (wf[:, None] * tj))
    return A


@pytest.mark.parametrize("n,k,lohi", [((1, 1, 1), 1, None), ((2, 1, 1), 2, None), ((2, 2, 1), 1, None),
                                      ((1, 2, 2), 2, ((0.0, -1.0, 0.5), (1.0, 2.0, 3.0))),
                                      ((3, 1, 2), 3, ((0.0, 0.0, 0.0), (1.5, 0.7, 2.0)))])
def test_projection_matches_brute_force_assembly(n, k, lohi):
    """The oracle's M + A_D + A_C equals the global matrix built pair by pair
    from the three bilinear forms, with cell-varying penalty parameters (one
    cell per direction and non-cubic cells included)."""
    m = dg.Mesh(n) if lohi is None else dg.Mesh(n, lo=lohi[0], hi=lohi[1])
    s = dg.Space(m, k)
    rng = np.random.default_rng(13)
    td, tc = rng.uniform(0.1, 1.0, m.E), rng.uniform(0.1, 1.0, m.E)
    B = _brute_force_projection(m, k, td, tc)
    U = rand((3, m.E, s.ndofs_cell), 14)
    y = B @ U.ravel()
    assert np.max(np.abs(dg.Projection(s, td, tc).apply(U).ravel() - y)) <= 1e-12 * np.max(np.abs(y))
