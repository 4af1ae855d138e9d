"""GPU vs oracle parity of the FP64 operators through the C ABI.

Bar: relative max-norm error <= 1e-12 (FP64 operators).  Cases span several
blocks of cells, ragged meshes (odd and unequal n), n = 1 (a cell is its own
periodic neighbour), non-cubic cells, a non-default penalty factor, and the
degree range k = 1..11.
"""
import numpy as np
import pytest
import torch

from oracle import dg, rules
from tests.gpu_common import build_lib, context, dev, host, random_field, rel_err, tgv_field

pytestmark = pytest.mark.gpu
TOL = 1e-12

LAP_CASES = [
    ((4, 4, 4), 3, {}),                                   # the 4^3, k=3 parity case
    ((3, 2, 5), 2, {}),
    ((1, 1, 1), 3, {}),
    ((2, 3, 1), 5, {"penalty_factor": 2.5}),
    ((5, 4, 3), 1, {}),
    ((3, 2, 2), 7, {"lo": (0.0, -1.0, 0.0), "hi": (1.0, 2.0, 0.5)}),
    ((2, 2, 2), 11, {}),
    ((7, 3, 2), 4, {}),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


def _mesh(n, kw):
    return dg.Mesh(n, kw.get("lo", (-np.pi,) * 3), kw.get("hi", (np.pi,) * 3))


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k,kw", LAP_CASES)
def test_laplace(n, k, kw, mode):
    """mode 0: native FP64; mode 1: double-float; mode 2: triple-float
    (FP32 pipe)."""
    ctx = context(n, k, k, mg_precision=0, fp64_mode=mode, **kw)
    s = dg.Space(_mesh(n, kw), k)
    x = random_field(s, 1, 0)
    ref = dg.Laplace(s, kw.get("penalty_factor", 1.0)).apply(x)
    y = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.vmult_laplace(y, dev(x), space=0)
    assert rel_err(host(y), ref) <= TOL
    # the diagonal of the same operator
    d = torch.empty_like(y)
    ctx.laplace_diagonal(d, space=0)
    assert rel_err(host(d), dg.Laplace(s, kw.get("penalty_factor", 1.0)).diagonal()) <= TOL


def test_laplace_pressure_space():
    n, ku = (3, 4, 2), 4
    ctx = context(n, ku, mg_precision=0)
    s = dg.Space(dg.Mesh(n), ku - 1)
    x = random_field(s, 1, 3)
    y = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.vmult_laplace(y, dev(x), space=1)
    assert rel_err(host(y), dg.Laplace(s).apply(x)) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k,kw", LAP_CASES[:6])
def test_mass_and_inverse(n, k, kw, mode):
    ctx = context(n, k, k, mg_precision=0, fp64_mode=mode, **kw)
    s = dg.Space(_mesh(n, kw), k)
    M = dg.Mass(s)
    for ncomp in (1, 3):
        x = random_field(s, ncomp, 1)
        y = torch.empty(x.size, dtype=torch.float64, device="cuda")
        ctx.vmult_mass(y, dev(x), ncomp=ncomp, space=0)
        assert rel_err(host(y), M.apply(x)) <= TOL
        ctx.apply_inverse_mass(y, dev(x), ncomp=ncomp, space=0)
        assert rel_err(host(y), M.apply_inverse(x)) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k", [((3, 2, 4), 3), ((2, 2, 3), 5), ((1, 2, 1), 2)])
def test_viscous_and_helmholtz(n, k, mode):
    nu = 1.0 / 1600
    ctx = context(n, k, mg_precision=0, nu=nu, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = random_field(s, 3, 2)
    y = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vmult_viscous(y, dev(u))
    assert rel_err(host(y), dg.Viscous(s, nu).apply(u)) <= TOL
    mf = 1.5 / 1e-3
    ctx.vmult_helmholtz(y, dev(u), mf)
    assert rel_err(host(y), dg.Helmholtz(s, nu, mf).apply(u)) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,ku", [((3, 2, 4), 3), ((2, 2, 2), 5), ((1, 2, 3), 2), ((2, 1, 1), 11),
                                  ((4, 4, 4), 4)])
def test_divergence_gradient(n, ku, mode):
    ctx = context(n, ku, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    su, sp = dg.Space(m, ku), dg.Space(m, ku - 1)
    u = random_field(su, 3, 4)
    p = random_field(sp, 1, 5)
    y = torch.empty(sp.size, dtype=torch.float64, device="cuda")
    ctx.vmult_divergence(y, dev(u))
    assert rel_err(host(y), dg.Divergence(su, sp).apply(u)) <= TOL
    g = torch.empty(3 * su.size, dtype=torch.float64, device="cuda")
    ctx.vmult_gradient(g, dev(p))
    assert rel_err(host(g), dg.Gradient(su, sp).apply(p)) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k,field", [((4, 4, 4), 3, "tgv"), ((3, 2, 5), 2, "rand"),
                                       ((2, 2, 2), 5, "rand"), ((1, 1, 2), 1, "rand"),
                                       ((2, 1, 1), 11, "tgv"), ((2, 3, 2), 7, "tgv"),
                                       ((5, 3, 2), 4, "tgv"), ((2, 2, 1), 9, "rand"),
                                       ((3, 3, 3), 3, "rand"), ((3, 1, 1), 1, "tgv"),
                                       ((2, 1, 2), 6, "tgv"), ((1, 2, 2), 8, "rand"),
                                       ((2, 2, 1), 10, "tgv")])
def test_convective(n, k, field, mode):
    """mode 0: native FP64; mode 1: double-float arithmetic (FP32 pipe).  Odd
    cell counts (27, 3) leave the last two-cell group of the k = 1 and k = 3
    kernels half empty."""
    ctx = context(n, k, max(k - 1, 1), mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-3, 0) if field == "tgv" else random_field(s, 3, 6)
    ref = dg.Convective(s).apply(u)
    y = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vmult_convective(y, dev(u))
    assert rel_err(host(y), ref) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k", [((3, 2, 2), 3), ((2, 3, 1), 5), ((2, 1, 2), 7), ((2, 2, 1), 9), ((2, 1, 1), 11)])
def test_convective_k_plus_1_points(n, k, mode):
    """The convective term with k + 1 Gauss points per direction instead of
    the 3/2 rule (n_q_conv = k + 1): the kernels' layouts without paired
    planes, the k = 9 cell kernel in its phase-aliased layout, and in mode 2
    the native kernels (the FP64-wide arrangements cover the 3/2 rule)."""
    ctx = context(n, k, k - 1, mg_precision=0, fp64_mode=mode, n_q_conv=k + 1)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-3, 1) if k % 2 else random_field(s, 3, 7)
    ref = dg.Convective(s, nq=k + 1).apply(u)
    y = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vmult_convective(y, dev(u))
    assert rel_err(host(y), ref) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k", [((3, 2, 2), 3), ((2, 1, 3), 2), ((1, 2, 1), 7), ((3, 1, 3), 3), ((3, 3, 1), 1)])
def test_convective_two_phases(n, k, mode):
    """Face kernel + cell kernel through the two-phase entry points give the
    one-call result exactly, and the oracle's result."""
    ctx = context(n, k, max(k - 1, 1), mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = dev(tgv_field(s, 1e-2, 3))
    rf = torch.empty(ctx.convective_face_size(), dtype=torch.float64, device="cuda")
    assert rf.numel() == 9 * s.mesh.E * (k + 1) ** 2
    y1 = torch.empty_like(u)
    y2 = torch.empty_like(u)
    ctx.convective_faces(rf, u)
    ctx.convective_cells(y1, u, rf)
    ctx.vmult_convective(y2, u)
    assert torch.equal(y1, y2)
    assert rel_err(host(y1), dg.Convective(s).apply(host(u).reshape(3, s.mesh.E, -1))) <= TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_convective_face_integrals_of_a_constant_field(mode):
    """For a constant velocity the LLF jump term vanishes and the face
    integral is u_c u_d h_t1 h_t2 omega_j1 omega_j2 (omega: integrals of the
    nodal basis on [0,1], i.e. the LGL weights), independent of the face."""
    n, k = (3, 2, 4), 3
    ctx = context(n, k, k - 1, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    uc = np.array([0.7, -0.4, 1.3])
    u = dev(np.repeat(uc, m.E * s.ndofs_cell))
    rf = torch.empty(ctx.convective_face_size(), dtype=torch.float64, device="cuda")
    ctx.convective_faces(rf, u)
    xg, wg = rules.gauss(k + 1)
    omega = wg @ rules.lagrange(rules.lgl_nodes(k), xg)[0]
    got = host(rf).reshape(3, m.E, 3, k + 1, k + 1)    # [d][e][c][j2][j1]
    for d in range(3):
        t1, t2 = [a for a in range(3) if a != d]
        ref = m.h[t1] * m.h[t2] * np.outer(omega, omega)   # [j2][j1] (symmetric)
        for c in range(3):
            want = uc[c] * uc[d] * ref
            assert np.max(np.abs(got[d, :, c] - want)) <= 1e-13 * np.max(np.abs(want))


def test_host_pointers_are_staged():
    """CPU tensors go through the library's staging buffers and give the same
    result as device tensors."""
    n, k = (3, 2, 2), 3
    ctx = context(n, k, mg_precision=0)
    s = dg.Space(dg.Mesh(n), k)
    x = random_field(s, 1, 9)
    yh = torch.empty(s.size, dtype=torch.float64)
    ctx.vmult_laplace(yh, torch.from_numpy(x.ravel().copy()), space=0)
    yd = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.vmult_laplace(yd, dev(x), space=0)
    assert np.array_equal(yh.numpy(), host(yd))


def test_alias_rejected():
    from paper_1802_01439_gb300 import DgnsError
    ctx = context((2, 2, 2), 2, mg_precision=0)
    x = torch.zeros(ctx.n_u, dtype=torch.float64, device="cuda")
    with pytest.raises(DgnsError):
        ctx.vmult_laplace(x, x, space=0)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n,k", [((8, 8, 8), 3), ((6, 4, 4), 5)])
def test_laplace_smooth_field(n, k, mode):
    """Smooth input: the stiffness sweeps cancel (L u ~ h^2 |terms|), the
    hardest case for the relative error."""
    ctx = context(n, k, k, mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    x = s.interpolate(lambda x, y, z: np.sin(x) * np.cos(y) * np.cos(2 * z) + 0.3)
    ref = dg.Laplace(s).apply(x)
    y = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.vmult_laplace(y, dev(x), space=0)
    assert rel_err(host(y), ref) <= TOL


def test_misaligned_vector_rejected():
    from paper_1802_01439_gb300 import DgnsError
    ctx = context((2, 2, 2), 3, 3, mg_precision=0)
    buf = torch.zeros(ctx.n_u + 1, dtype=torch.float64, device="cuda")
    y = torch.empty(ctx.n_u, dtype=torch.float64, device="cuda")
    with pytest.raises(DgnsError):
        ctx.vmult_laplace(y, buf[1:], space=0)


def test_pinned_host_pointers():
    """Pinned host tensors (staged like any host memory) give the device-tensor
    results, also through the two-phase convective entry points."""
    n, k = (3, 2, 2), 3
    ctx = context(n, k, k - 1, mg_precision=0, fp64_mode=1)
    s = dg.Space(dg.Mesh(n), k)
    u = torch.from_numpy(tgv_field(s, 1e-2, 2).ravel().copy())
    up = u.pin_memory()
    yp = torch.empty(u.numel(), dtype=torch.float64).pin_memory()
    yd = torch.empty(u.numel(), dtype=torch.float64, device="cuda")
    ctx.vmult_convective(yp, up)
    ctx.vmult_convective(yd, u.cuda())
    assert np.array_equal(yp.numpy(), host(yd))
    ctx.vmult_helmholtz(yp, up, 1500.0)
    ctx.vmult_helmholtz(yd, u.cuda(), 1500.0)
    assert np.array_equal(yp.numpy(), host(yd))
    rf = torch.empty(ctx.convective_face_size(), dtype=torch.float64).pin_memory()
    ctx.convective_faces(rf, up)
    ctx.convective_cells(yp, up, rf)
    ctx.vmult_convective(yd, u.cuda())
    assert np.array_equal(yp.numpy(), host(yd))


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scale", [1e-300, 1e-20, 1e-15, 1.0, 1e30, 1e35, 1e300])
def test_emulated_modes_across_the_fp64_range(scale, mode):
    """Double-float and triple-float values carry float's exponent; inputs
    whose largest entry lies outside the window the emulations keep to full
    precision are scaled by an exact power of two inside the call, so every
    scale FP64 holds gives the same relative accuracy (the previous build
    measured 1.8e-10 at 1e-20 without the scaling).  Linear operators: mass,
    inverse mass, Laplace, Helmholtz, divergence, gradient, projection."""
    n, k = (2, 3, 2), 3
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    s, sp = dg.Space(m, k), dg.Space(m, k - 1)
    x = scale * random_field(s, 3, 12)
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    ctx.vmult_mass(y, dev(x.ravel()), 3, 0)
    assert rel_err(host(y), dg.Mass(s).apply(x)) <= TOL
    ctx.apply_inverse_mass(y, dev(x.ravel()), 3, 0)
    assert rel_err(host(y), dg.Mass(s).apply_inverse(x)) <= TOL
    ctx.vmult_laplace(y[:s.size], dev(x[0].ravel()), space=0)
    assert rel_err(host(y[:s.size]), dg.Laplace(s).apply(x[0])) <= TOL
    ctx.vmult_helmholtz(y, dev(x.ravel()), 1500.0)
    assert rel_err(host(y), dg.Helmholtz(s, 1.0 / 1600, 1500.0).apply(x)) <= TOL
    d = torch.empty(sp.size, dtype=torch.float64, device="cuda")
    ctx.vmult_divergence(d, dev(x.ravel()))
    assert rel_err(host(d), dg.Divergence(s, sp).apply(x)) <= TOL
    p = scale * random_field(sp, 1, 13)
    ctx.vmult_gradient(y, dev(p.ravel()))
    assert rel_err(host(y), dg.Gradient(s, sp).apply(p)) <= TOL
    td, tc = np.full(m.E, 0.3), np.full(m.E, 0.2)
    ctx.vmult_projection(y, dev(x.ravel()), dev(td), dev(tc))
    assert rel_err(host(y), dg.Projection(s, td, tc).apply(x)) <= TOL


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scale", [1e-150, 1e-20, 1e20, 1e150])
def test_emulated_convective_across_the_fp64_range(scale, mode):
    """The convective term is quadratic: inputs are scaled into the window
    of the emulations and the result by the square of the factor, in the
    one-call form and in its two phases (face integrals, cell term)."""
    n, k = (2, 2, 3), 3
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = scale * tgv_field(s, 1e-2, 3)
    ref = dg.Convective(s).apply(u)
    y = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vmult_convective(y, dev(u.ravel()))
    assert rel_err(host(y), ref) <= TOL
    rf = torch.empty(ctx.convective_face_size(), dtype=torch.float64, device="cuda")
    ud = dev(u.ravel())
    ctx.convective_faces(rf, ud)
    ctx.convective_cells(y, ud, rf)
    assert rel_err(host(y), ref) <= TOL


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scale", [1e-250, 1e-20, 1e250])
def test_emulated_solves_across_the_fp64_range(scale, mode):
    """The Helmholtz and pressure solves scale the right-hand side into the
    window and the solution back: the solution of scale * b is scale times
    the solution of b."""
    n, k = (4, 4, 2), 3
    ctx = context(n, k, mg_precision=32, fp64_mode=mode)
    b = np.random.default_rng(14).uniform(-1, 1, 3 * ctx.n_u)
    x1, xs = (torch.zeros(3 * ctx.n_u, dtype=torch.float64, device="cuda") for _ in range(2))
    ctx.cg_invmass_solve(x1, dev(b), 100.0, rel_tol=1e-12)
    ctx.cg_invmass_solve(xs, dev(scale * b), 100.0, rel_tol=1e-12)
    assert rel_err(host(xs) / scale, host(x1)) <= 1e-11
    bp = b[:ctx.n_p] - b[:ctx.n_p].mean()
    p1, ps = (torch.zeros(ctx.n_p, dtype=torch.float64, device="cuda") for _ in range(2))
    ctx.cg_mg_solve(p1, dev(bp), rel_tol=1e-11)
    ctx.cg_mg_solve(ps, dev(scale * bp), rel_tol=1e-11)
    assert rel_err(host(ps) / scale, host(p1)) <= 1e-9


# ------------------------------------------ triple-float: FP64-wide accuracy
@pytest.mark.parametrize("n,k,field", [((4, 4, 4), 3, "rand"), ((3, 2, 2), 5, "rand"),
                                       ((2, 2, 1), 7, "rand"), ((8, 8, 8), 3, "smooth"),
                                       ((4, 4, 2), 5, "smooth")])
def test_triple_float_at_least_as_accurate_as_fp64(n, k, field):
    """Against the oracle evaluated in extended precision (np.longdouble, its
    own tables included), the triple-float SIPG operator (mode 2) is at least
    as accurate as native FP64 (mode 0): both use the same FP64-rounded 1D
    tables, so the difference is the arithmetic's own rounding.  Smooth fields
    (sin x cos y sin z) make the stiffness sweeps cancel.  Degrees up to 7: the
    extended-precision element matrices cost (k+1)^9 software-float
    operations on hosts where long double is binary128."""
    s = dg.Space(dg.Mesh(n), k)
    se = dg.Space(dg.Mesh(n, dtype=np.longdouble), k)
    if field == "rand":
        x = random_field(s, 1, 9)
    else:
        x = s.interpolate(lambda a, b, c: np.sin(a) * np.cos(b) * np.sin(c))
    ref = dg.Laplace(se).apply(x).astype(np.float64)
    errs = {}
    for mode in (0, 2):
        ctx = context(n, k, k, mg_precision=0, fp64_mode=mode)
        y = torch.empty(s.size, dtype=torch.float64, device="cuda")
        ctx.vmult_laplace(y, dev(x), space=0)
        errs[mode] = rel_err(host(y), ref)
    print("laplace %s k=%d: native %.2e, triple-float %.2e vs extended" % (field, k, errs[0], errs[2]))
    assert errs[2] <= TOL
    assert errs[2] <= 1.5 * errs[0] + 1e-16
