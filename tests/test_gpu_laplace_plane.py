"""The kernels of the FP32 SIPG level operator at k_p = 3 (Sec. 3.3: the
multigrid smoother's operator) against the FP64 oracle on every level of the
hierarchy: one thread per cell plane (256-bit or 128-bit accesses, the
z-direction as one or two reduce-scatters) and one thread per x-line, with the
plain, residual and Chebyshev epilogues.  Meshes of 5^3 and 12^3 cells give
ragged last blocks (125, 27 cells); vectors offset by 16 bytes are not
32-byte aligned, so the 256-bit variants hand them to the line kernel.
Bar: relative max-norm error <= 1e-5 (FP32 rounding of ~30 terms per node)."""
import numpy as np
import pytest
import torch

from oracle import dg, mg
from tests.gpu_common import build_lib, context, host, rel_err

pytestmark = pytest.mark.gpu

KP = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


def _vec(a, offset):
    """FP32 device copy of a, starting `offset` floats into its allocation."""
    buf = torch.zeros(a.size + offset, dtype=torch.float32, device="cuda")
    v = buf[offset:]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    return v


def _empty(n, offset):
    return torch.full((n + offset,), np.nan, dtype=torch.float32, device="cuda")[offset:]


@pytest.mark.parametrize("offset", [0, 4])
@pytest.mark.parametrize("variant", [-1, 0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [5, 12, 16])
def test_level_operator_kernels(n, variant, offset):
    ctx = context(n, KP + 1, KP)
    lib = ctx.lib
    assert lib.dgns_debug_laplace_f32_kernel(variant) == 0
    try:
        H = mg.Hierarchy(dg.Mesh(n), KP, coarse_n=2)
        assert ctx.mg_info()["levels"] == len(H.levels)
        rng = np.random.default_rng(100 + n)
        for lvl, L in enumerate(H.levels):
            s = L["space"]
            A = L["op"].apply
            x = rng.uniform(-1, 1, s.size).astype(np.float32)
            xp = rng.uniform(-1, 1, s.size).astype(np.float32)
            b = rng.uniform(-1, 1, s.size).astype(np.float32)
            X = x.astype(np.float64).reshape(s.mesh.E, -1)
            Ax = A(X)
            y = _empty(s.size, offset)
            ctx.vmult_laplace_f32(y, _vec(x, offset), lvl)
            assert rel_err(host(y), Ax) <= 1e-5
            # Chebyshev step dst = x + c1 (x - xprev) + c2 D^-1 (b - A x)
            c1, c2 = 0.37, 0.021
            dinv = L["inv_diag"].reshape(s.mesh.E, -1)
            ref = X + c1 * (X - xp.astype(np.float64).reshape(X.shape)) + \
                c2 * dinv * (b.astype(np.float64).reshape(X.shape) - Ax)
            ctx.mg_chebyshev_step_f32(y, _vec(x, offset), _vec(xp, offset), _vec(b, offset), c1, c2, lvl)
            assert rel_err(host(y), ref) <= 1e-5
            # c1 = 0 with no previous iterate (the first step from a guess)
            ref0 = X + c2 * dinv * (b.astype(np.float64).reshape(X.shape) - Ax)
            ctx.mg_chebyshev_step_f32(y, _vec(x, offset), None, _vec(b, offset), 0.0, c2, lvl)
            assert rel_err(host(y), ref0) <= 1e-5
        assert lib.dgns_debug_laplace_f32_timeouts() == 0
    finally:
        lib.dgns_debug_laplace_f32_kernel(0)


def test_kernel_choice_rejects_unknown_variants():
    ctx = context(4, KP + 1, KP)
    assert ctx.lib.dgns_debug_laplace_f32_kernel(6) != 0
    assert ctx.lib.dgns_debug_laplace_f32_kernel(-2) != 0
    assert ctx.lib.dgns_debug_laplace_f32_kernel(0) == 0


def test_packed_scalar_and_staged_kernels_agree_bitwise():
    """The packed FP32x2 arithmetic performs every element's operations in
    the scalar order, and the staged kernel runs the same arithmetic: the
    three give identical bits (16^3 cells: the staged kernel applies)."""
    n = 16
    ctx = context(n, KP + 1, KP)
    lib = ctx.lib
    lvl = ctx.mg_info()["levels"] - 1
    rng = np.random.default_rng(7)
    size = n ** 3 * (KP + 1) ** 3
    x = _vec(rng.uniform(-1, 1, size), 0)
    xp = _vec(rng.uniform(-1, 1, size), 0)
    b = _vec(rng.uniform(-1, 1, size), 0)
    outs = []
    try:
        for v in (1, 2, 4):
            assert lib.dgns_debug_laplace_f32_kernel(v) == 0
            y = _empty(size, 0)
            ctx.mg_chebyshev_step_f32(y, x, xp, b, 0.37, 0.021, lvl)
            z = _empty(size, 0)
            ctx.vmult_laplace_f32(z, x, lvl)
            outs.append((host(y), host(z)))
        assert lib.dgns_debug_laplace_f32_timeouts() == 0
    finally:
        lib.dgns_debug_laplace_f32_kernel(0)
    for y, z in outs[1:]:
        assert np.array_equal(y, outs[0][0]) and np.array_equal(z, outs[0][1])
