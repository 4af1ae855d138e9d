"""GPU vs oracle parity of the projection-step operator with the divergence
and continuity penalty terms (Sec. 3.2) and of its penalty parameters, and the
inverse-mass-preconditioned CG solve of the projection system (Sec. 3.3)."""
import numpy as np
import pytest
import torch

from oracle import dg, solvers
from tests.gpu_common import build_lib, context, dev, host, random_field, rel_err, tgv_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


@pytest.mark.parametrize("n,k", [((3, 2, 4), 3), ((2, 2, 2), 2), ((1, 2, 3), 4), ((2, 1, 2), 7),
                                 ((2, 1, 1), 9), ((1, 2, 1), 11)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_penalty_parameters(n, k, mode):
    """mode 1: interpolation and norm in double-float (with its square root)."""
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    s = dg.Space(dg.Mesh(n), k)
    u = tgv_field(s, 1e-2, 1)
    td, tc = ctx.penalty_parameters(dev(u.ravel()), 1e-3, zeta_d=1.0, zeta_c=0.7)
    rd, rc = dg.penalty_parameters(s, u, 1e-3, zeta_d=1.0, zeta_c=0.7)
    assert rel_err(host(td), rd) <= 1e-12 and rel_err(host(tc), rc) <= 1e-12


@pytest.mark.parametrize("n,k", [((3, 2, 4), 3), ((2, 2, 2), 2), ((1, 2, 3), 4), ((2, 1, 2), 7),
                                 ((4, 3, 2), 5), ((2, 1, 1), 6), ((1, 2, 2), 8), ((2, 1, 2), 9),
                                 ((2, 2, 1), 10), ((1, 1, 2), 11)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_projection_operator(n, k, mode):
    """mode 0: native FP64; mode 1: double-float arithmetic; mode 2 runs the
    projection kernels natively."""
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    rng = np.random.default_rng(3)
    td, tc = rng.uniform(0.1, 1.0, m.E), rng.uniform(0.1, 1.0, m.E)
    u = random_field(s, 3, 8)
    y = torch.empty(u.size, dtype=torch.float64, device="cuda")
    ctx.vmult_projection(y, dev(u.ravel()), dev(td), dev(tc))
    assert rel_err(host(y), dg.Projection(s, td, tc).apply(u)) <= 1e-12


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_projection_solve(mode):
    n, k, dt = (4, 3, 4), 3, 1e-3
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    u = tgv_field(s, 1e-3, 2)
    td, tc = dg.penalty_parameters(s, u, dt)
    b = np.random.default_rng(4).uniform(-1, 1, 3 * s.size)
    x = torch.zeros(3 * s.size, dtype=torch.float64, device="cuda")
    info = ctx.cg_projection_solve(x, dev(b), dev(td), dev(tc), rel_tol=1e-12)
    assert info["rc"] == 0 and info["iterations"] <= 20
    P = dg.Projection(s, td, tc)
    assert solvers.relative_residual(lambda v: P.apply(v.reshape(3, m.E, -1)).ravel(), host(x), b) <= 2e-12


@pytest.mark.parametrize("n,k", [((3, 2, 4), 3), ((2, 3, 1), 5), ((1, 2, 2), 9), ((2, 1, 1), 11)])
@pytest.mark.parametrize("mode", [0, 1])
def test_projection_terms(n, k, mode):
    """Each term in its own pass (the operator-by-operator evaluation): M by
    the mass kernel, A_D and A_C by their own kernels, against the oracle's
    terms; their sum equals the fused operator."""
    from paper_1802_01439_gb300 import _lib
    ctx = context(n, k, mg_precision=0, fp64_mode=mode)
    m = dg.Mesh(n)
    s = dg.Space(m, k)
    rng = np.random.default_rng(5)
    td, tc = rng.uniform(0.1, 1.0, m.E), rng.uniform(0.1, 1.0, m.E)
    u = random_field(s, 3, 9)
    P = dg.Projection(s, td, tc)
    total = torch.zeros(u.size, dtype=torch.float64, device="cuda")
    for terms, name in ((_lib.PROJ_MASS, "M"), (_lib.PROJ_DIV, "D"), (_lib.PROJ_CONT, "C")):
        y = torch.empty(u.size, dtype=torch.float64, device="cuda")
        ctx.vmult_projection(y, dev(u.ravel()), dev(td) if name != "C" else None,
                             dev(tc) if name != "D" else None, terms=terms)
        assert rel_err(host(y), P.apply(u, terms=name)) <= 1e-12, name
        total += y
    fused = torch.empty_like(total)
    ctx.vmult_projection(fused, dev(u.ravel()), dev(td), dev(tc))
    assert rel_err(host(total), host(fused)) <= 1e-12


def test_projection_terms_rejected():
    from paper_1802_01439_gb300 import DgnsError
    ctx = context((1, 1, 1), 3, mg_precision=0)
    x = torch.zeros(3 * ctx.n_u, dtype=torch.float64, device="cuda")
    t = torch.ones(1, dtype=torch.float64, device="cuda")
    with pytest.raises(DgnsError):
        ctx.vmult_projection(torch.empty_like(x), x, t, t, terms=3)
