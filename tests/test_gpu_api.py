"""GPU tests of the C-ABI entry points that the operator tests reach only
indirectly: stream selection, the vector helpers, sizes and destruction."""
import numpy as np
import pytest
import torch

from oracle import dg
from tests.gpu_common import build_lib, context, dev, host, random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


def test_sizes():
    ctx = context((3, 2, 5), 4, 2, mg_precision=0)
    assert ctx.n_u == 30 * 5 ** 3 and ctx.n_p == 30 * 3 ** 3


def test_set_stream_runs_operators_and_solves_on_the_new_stream():
    """The same operator and the same multigrid-preconditioned solve (its
    V-cycle replayed from a CUDA graph) give bit-identical results on the
    stream given at creation and on a stream set later (fixed-order
    reductions)."""
    n, k = (4, 4, 4), 3
    ctx = context(n, k, mg_precision=32)
    s = dg.Space(dg.Mesh(n), k - 1)
    x = dev(random_field(s, 1, 1))
    b = dev(random_field(s, 1, 2))
    b -= b.mean()
    y0 = torch.empty_like(x)
    ctx.vmult_laplace(y0, x)
    p0 = torch.zeros_like(b)
    ctx.cg_mg_solve(p0, b)
    torch.cuda.synchronize()
    s2 = torch.cuda.Stream()
    ctx.set_stream(s2)
    with torch.cuda.stream(s2):
        y1 = torch.empty_like(x)
        ctx.vmult_laplace(y1, x)
        p1 = torch.zeros_like(b)
        ctx.cg_mg_solve(p1, b)
    s2.synchronize()
    assert torch.equal(y0, y1)
    assert torch.equal(p0, p1)


def test_axpby_and_dot():
    ctx = context((2, 2, 2), 2, mg_precision=0)
    rng = np.random.default_rng(3)
    xn, yn = rng.uniform(-1, 1, 1001), rng.uniform(-1, 1, 1001)
    x, y = dev(xn), dev(yn)
    ctx.axpby(y, x, 0.75, -1.5)
    assert np.max(np.abs(host(y) - (0.75 * xn - 1.5 * yn))) <= 1e-15
    # b = 0 ignores the prior contents of y, NaN included
    y.fill_(float("nan"))
    ctx.axpby(y, x, 2.0, 0.0)
    assert np.array_equal(host(y), 2.0 * xn)
    # x may be y
    ctx.axpby(y, y, 0.5, 0.25)
    assert np.max(np.abs(host(y) - 0.75 * (2.0 * xn))) <= 1e-15
    d = ctx.dot(x, dev(yn))
    assert abs(d - float(np.dot(xn, yn))) <= 1e-14 * np.sum(np.abs(xn * yn))
    assert ctx.dot(x, dev(yn)) == d                  # fixed-order reduction: reproducible


def test_destroyed_context_rejects_calls():
    from paper_1802_01439_gb300 import DgnsError
    ctx = context((2, 2, 2), 2, mg_precision=0)
    x = torch.zeros(ctx.n_p, dtype=torch.float64, device="cuda")
    ctx.close()
    ctx.close()                                       # idempotent
    with pytest.raises(DgnsError):
        ctx.vmult_laplace(torch.empty_like(x), x)


def test_failed_create_frees_everything():
    """Each device allocation of a context creation (tables, reduction
    buffers, CG vectors, multigrid levels, the eigenvalue estimate's work
    vector) is made to fail in turn: every such creation returns
    DGNS_ERR_OOM, hands back no context and leaves no allocation behind;
    the first n past the last allocation creates the context normally."""
    import gc
    from paper_1802_01439_gb300 import DgnsError, _lib
    lib = _lib.load()
    # contexts of earlier tests held in reference cycles must not be freed
    # while the live count is being compared
    gc.collect()
    gc.disable()
    try:
        _fail_each_allocation(lib, DgnsError, _lib)
    finally:
        gc.enable()


def _fail_each_allocation(lib, DgnsError, _lib):
    base = lib.dgns_debug_live_allocations()
    ctx = context((4, 4, 4), 3, mg_precision=32)
    kept = lib.dgns_debug_live_allocations() - base
    ctx.close()
    assert lib.dgns_debug_live_allocations() == base and kept > 10
    n = 1
    try:
        while n < 200:
            lib.dgns_debug_fail_alloc(n)
            try:
                ctx = context((4, 4, 4), 3, mg_precision=32)
            except DgnsError as err:
                assert err.code == _lib.DGNS_ERR_OOM, err
                assert lib.dgns_debug_live_allocations() == base, n
                n += 1
                continue
            break
    finally:
        lib.dgns_debug_fail_alloc(0)
    assert n > kept                     # every kept allocation failed once
    assert lib.dgns_debug_live_allocations() == base + kept
    ctx.close()
    assert lib.dgns_debug_live_allocations() == base
