"""GPU vs oracle parity of the multigrid components and the solvers.

FP32 level operators and transfers: relative max-norm error <= 1e-5 against
the FP64 oracle on the same (FP32-rounded) input.  The FP64 V-cycle matches
the oracle's V-cycle to 1e-11 given the same eigenvalue bounds; the FP32
V-cycle to 1e-4 (Chebyshev polynomials of degree 5/20 amplify the FP32
rounding of each level operator by at most their maximum on the smoothing
interval, a few hundred at worst).  Solves are checked through the oracle's
own FP64 residual.
"""
import numpy as np
import pytest
import torch

from oracle import dg, mg, solvers
from tests.gpu_common import build_lib, context, dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


def rand32(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, n).astype(np.float32)


@pytest.mark.parametrize("n,kp", [(8, 3), (4, 2), (6, 5)])
def test_level_operators_fp32(n, kp):
    ctx = context(n, kp + 1, kp)
    info = ctx.mg_info()
    H = mg.Hierarchy(dg.Mesh(n), kp, coarse_n=2)
    assert info["levels"] == len(H.levels)
    for lvl, L in enumerate(H.levels):
        s = L["space"]
        x = rand32(s.size, lvl)
        y = torch.empty(s.size, dtype=torch.float32, device="cuda")
        ctx.vmult_laplace_f32(y, dev(x, torch.float32), lvl)
        ref = L["op"].apply(x.astype(np.float64).reshape(s.mesh.E, -1))
        assert rel_err(host(y), ref) <= 1e-5
    for lvl in range(len(H.levels) - 1):
        T = H.transfers[lvl]
        xc = rand32(T.cs.size, 10 + lvl)
        xf = torch.empty(T.fs.size, dtype=torch.float32, device="cuda")
        ctx.mg_prolongate_f32(xf, dev(xc, torch.float32), lvl)
        assert rel_err(host(xf), T.prolongate(xc.astype(np.float64).reshape(T.cs.mesh.E, -1))) <= 1e-5
        xf0 = rand32(T.fs.size, 20 + lvl)
        yc = torch.empty(T.cs.size, dtype=torch.float32, device="cuda")
        ctx.mg_restrict_f32(yc, dev(xf0, torch.float32), lvl)
        assert rel_err(host(yc), T.restrict(xf0.astype(np.float64).reshape(T.fs.mesh.E, -1))) <= 1e-5


@pytest.mark.parametrize("n,kp", [(8, 3), (6, 2), (4, 5)])
def test_chebyshev_step_fp32(n, kp):
    """The fused FP32 smoother step (the level operator with its Chebyshev
    epilogue, as the V-cycle runs it) against the oracle's Chebyshev
    iteration (Saad, Alg. 12.1) on the finest level, same interval:
    one step from x0 at 1e-5, and five steps with the three-term
    coefficients at 1e-4."""
    ctx = context(n, kp + 1, kp)
    lvl = ctx.mg_info()["levels"] - 1
    lam = ctx.mg_info()["lambda_max"][lvl]
    s = dg.Space(dg.Mesh(n), kp)
    L = dg.Laplace(s)
    inv_diag = 1.0 / L.diagonal()
    A = L.apply
    x0 = rand32(s.size, 31)
    b = rand32(s.size, 32)
    X0, B = x0.astype(np.float64).reshape(s.mesh.E, -1), b.astype(np.float64).reshape(s.mesh.E, -1)
    rng_, lmin = 20.0, lam / 20.0
    theta, delta = 0.5 * (lam + lmin), 0.5 * (lam - lmin)
    sigma = theta / delta
    f32 = dict(dtype=torch.float32, device="cuda")
    xs = [dev(x0, torch.float32)]
    bd = dev(b, torch.float32)
    y = torch.empty(s.size, **f32)
    ctx.mg_chebyshev_step_f32(y, xs[0], None, bd, 0.0, 1.0 / theta, lvl)
    ref1 = mg.chebyshev(A, inv_diag, B, X0, lam, rng_, 1)
    assert rel_err(host(y), ref1) <= 1e-5
    xs.append(y)
    rho = 1.0 / sigma
    for k in range(1, 5):
        rnew = 1.0 / (2.0 * sigma - rho)
        c1, c2 = rnew * rho, 2.0 * rnew / delta
        rho = rnew
        nxt = torch.empty(s.size, **f32)
        ctx.mg_chebyshev_step_f32(nxt, xs[-1], xs[-2], bd, c1, c2, lvl)
        xs.append(nxt)
    ref5 = mg.chebyshev(A, inv_diag, B, X0, lam, rng_, 5)
    assert rel_err(host(xs[-1]), ref5) <= 1e-4


def test_lambda_estimates_bound_the_spectrum():
    n, kp = 4, 2
    ctx = context(n, kp + 1, kp)
    lam = ctx.mg_info()["lambda_max"]
    H = mg.Hierarchy(dg.Mesh(n), kp, coarse_n=2)
    for L, l_gpu in zip(H.levels, lam):
        A = L["op"].matrix()
        d = np.sqrt(L["inv_diag"].ravel())
        true = np.linalg.eigvalsh(d[:, None] * A * d[None, :])[-1]
        assert true <= l_gpu <= 1.3 * true


@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (32, 1e-4)])
def test_vcycle_matches_oracle(prec, tol):
    n, kp = 8, 3
    ctx = context(n, kp + 1, kp, mg_precision=prec)
    lam = ctx.mg_info()["lambda_max"]
    H = mg.Hierarchy(dg.Mesh(n), kp, coarse_n=2)
    s = H.levels[-1]["space"]
    r = np.random.default_rng(7).uniform(-1, 1, s.size)
    z = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.mg_vcycle(z, dev(r))
    ref = H.vcycle(r.reshape(s.mesh.E, -1), lam, degree=5, smoothing_range=20.0, coarse_iters=20)
    assert rel_err(host(z), ref) <= tol


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,kp", [(8, 3), (4, 2), ((4, 8, 4), 3)])
def test_cg_mg_solve(prec, n, kp):
    ctx = context(n, kp + 1, kp, mg_precision=prec)
    s = dg.Space(dg.Mesh(n), kp)
    b = solvers.mean_free(np.random.default_rng(11).uniform(-1, 1, s.size))
    x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    info = ctx.cg_mg_solve(x, dev(b), rel_tol=1e-10)
    assert info["rc"] == 0 and info["rel_res"] <= 1e-10
    assert info["iterations"] <= 30
    L = dg.Laplace(s)
    assert solvers.relative_residual(lambda v: L.apply(v.reshape(s.mesh.E, -1)).ravel(),
                                     host(x), b) <= 1.5e-10


@pytest.mark.parametrize("prec", [32, 64])
def test_cg_mg_solve_without_mean_projection(prec):
    """project_mean = 0: the V-cycle output keeps its constant component (the
    null space of the periodic operator), so the solve still converges to the
    relative tolerance and its solution differs from the projected one by a
    constant only (the V-cycle exit then widens and sums (r, z) unshifted)."""
    n, kp = 8, 3
    ctx = context(n, kp + 1, kp, mg_precision=prec)
    s = dg.Space(dg.Mesh(n), kp)
    b = solvers.mean_free(np.random.default_rng(12).uniform(-1, 1, s.size))
    xs = []
    for pm in (1, 0):
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        info = ctx.cg_mg_solve(x, dev(b), rel_tol=1e-10, project_mean=pm)
        assert info["rc"] == 0 and info["rel_res"] <= 1e-10 and info["iterations"] <= 30
        xs.append(host(x))
    L = dg.Laplace(s)
    assert solvers.relative_residual(lambda v: L.apply(v.reshape(s.mesh.E, -1)).ravel(), xs[1], b) <= 1.5e-10
    d = (xs[1] - xs[1].mean()) - (xs[0] - xs[0].mean())
    assert np.max(np.abs(d)) <= 1e-6 * np.max(np.abs(xs[0]))


def test_cg_not_converged_is_reported():
    ctx = context(4, 3, 2)
    s = dg.Space(dg.Mesh(4), 2)
    b = solvers.mean_free(np.random.default_rng(1).uniform(-1, 1, s.size))
    x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    info = ctx.cg_mg_solve(x, dev(b), raise_on_error=False, rel_tol=1e-14, max_iter=2)
    assert info["rc"] == 4 and info["iterations"] == 2


def test_cg_nonfinite_is_reported():
    ctx = context(4, 3, 2)
    b = torch.full((ctx.n_p,), float("nan"), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = ctx.cg_mg_solve(x, b, raise_on_error=False)
    assert info["rc"] == 5


def test_helmholtz_invmass_cg():
    n, k = (4, 3, 4), 3
    nu, mf = 1.0 / 1600, 1.5 / 1e-3
    ctx = context(n, k, mg_precision=0, nu=nu)
    s = dg.Space(dg.Mesh(n), k)
    b = np.random.default_rng(3).uniform(-1, 1, 3 * s.size)
    x = torch.zeros(3 * s.size, dtype=torch.float64, device="cuda")
    info = ctx.cg_invmass_solve(x, dev(b), mf, rel_tol=1e-12)
    assert info["rc"] == 0 and info["iterations"] <= 15
    Hm = dg.Helmholtz(s, nu, mf)
    res = solvers.relative_residual(lambda v: Hm.apply(v.reshape(3, s.mesh.E, -1)).ravel(), host(x), b)
    assert res <= 2e-12


@pytest.mark.parametrize("kp", [2, 3])
def test_cg_mg_iterations_are_mesh_independent(kp):
    """Sec. 3.3: with the multigrid V-cycle as preconditioner the pressure CG
    needs a number of iterations that does not grow under mesh refinement
    (the paper reports 6-12 at relative tolerance 1e-6 over its refinement
    levels).  Mean-free random right-hand side, zero initial guess,
    relative tolerance 1e-6, FP32 V-cycle, 8^3, 16^3 and 32^3 cells (3, 4
    and 5 levels): the counts differ by at most 2 and none exceeds 12."""
    its = []
    for n in (8, 16, 32):
        ctx = context(n, kp + 1, kp, mg_precision=32)
        s = dg.Space(dg.Mesh(n), kp)
        b = solvers.mean_free(np.random.default_rng(12).uniform(-1, 1, s.size))
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        info = ctx.cg_mg_solve(x, dev(b), rel_tol=1e-6)
        assert info["rc"] == 0 and info["rel_res"] <= 1e-6
        its.append(info["iterations"])
    assert max(its) - min(its) <= 2 and max(its) <= 12, its


def test_widen_f32_is_exact():
    """The FP32 -> FP64 conversion at the V-cycle's exit (done on the bit
    patterns for normal floats and zeros) gives the IEEE 754 value of every
    float: random normal floats over the whole exponent range, signed zeros,
    the extreme normals, subnormals, infinities and a NaN."""
    ctx = context(2, 2)
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, 1.0, -1.0, np.finfo(np.float32).max, -np.finfo(np.float32).max,
                        np.finfo(np.float32).tiny, -np.finfo(np.float32).tiny, 1e-40, -3e-45,
                        np.inf, -np.inf, np.nan], dtype=np.float32)
    x = np.concatenate([bits.view(np.float32), special])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty(x.size, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert ctx.lib.dgns_debug_widen_f32(xd.data_ptr(), yd.data_ptr(), x.size) == 0
    y = yd.cpu().numpy()
    ref = x.astype(np.float64)
    fin = ~np.isnan(ref)
    assert np.array_equal(y[fin].view(np.uint64), ref[fin].view(np.uint64))
    assert np.all(np.isnan(y[~fin]))
    assert ctx.lib.dgns_debug_widen_f32(xd.data_ptr(), yd.data_ptr(), -1) != 0
    assert ctx.lib.dgns_debug_widen_f32(xd.data_ptr(), yd.data_ptr(), 0) == 0
