"""The allocation-free Helmholtz CG entry point (dgns_cg_invmass_solve_noalloc)
gives the same solution as dgns_cg_invmass_solve, and allocates nothing.

Callers that cannot let a library allocate device memory (applications whose
device memory belongs to their own pool, real-time loops that must not risk
allocation latency or failure mid-step) use this variant; its work vectors
live in a fixed array inside the library.  Two calls in a row with different
right-hand sides check that the shared scratch carries no state from one call
to the next.  This file sorts last so that a run stopping at its first
failure has run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests.gpu_common import build_lib, context

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _solve(lib, ctx, fn, b, mf, x=None, **kw):
    from paper_1802_01439_gb300 import _lib
    x = torch.zeros_like(b) if x is None else x
    prm = ctx.solve_params(rel_tol=1e-12, **kw)
    info = _lib.SolveInfo()
    rc = getattr(lib, fn)(ctx.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                          ctypes.c_double(mf), ctypes.byref(prm), ctypes.byref(info))
    torch.cuda.synchronize()
    return rc, x.cpu().numpy(), info


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_allocating_solve(mode):
    """Native FP64 (mode 0) and double-float (mode 1) matvecs: both solves
    use the context's arithmetic."""
    build_lib()
    from paper_1802_01439_gb300 import _lib
    lib = _lib.load()
    ctx = context((4, 3, 5), 3, mg_precision=0, nu=1.0 / 1600, fp64_mode=mode)
    mf = 1.5 / 1e-3
    for seed in (1, 2):
        b = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, 3 * ctx.n_u)).cuda()
        rc0, x0, i0 = _solve(lib, ctx, "dgns_cg_invmass_solve", b, mf)
        rc1, x1, i1 = _solve(lib, ctx, "dgns_cg_invmass_solve_noalloc", b, mf)
        assert rc0 == 0 and rc1 == 0
        assert i1.iterations == i0.iterations and i1.rel_res <= 1e-12
        assert np.max(np.abs(x1 - x0)) <= TOL * np.max(np.abs(x0))


def test_noalloc_initial_guess_matches_allocating_solve():
    """With use_initial_guess the residual is formed from the caller's x
    (SIPG matvec into the shared scratch, then axpby and dot there)."""
    build_lib()
    from paper_1802_01439_gb300 import _lib
    lib = _lib.load()
    ctx = context((3, 4, 2), 4, mg_precision=0, nu=1.0 / 1600)
    mf = 1.5 / 1e-3
    rng = np.random.default_rng(7)
    b = torch.from_numpy(rng.uniform(-1, 1, 3 * ctx.n_u)).cuda()
    guess = rng.uniform(-1, 1, 3 * ctx.n_u) * 1e-3
    xa = torch.from_numpy(guess.copy()).cuda()
    xb = torch.from_numpy(guess.copy()).cuda()
    rc0, x0, i0 = _solve(lib, ctx, "dgns_cg_invmass_solve", b, mf, x=xa, use_initial_guess=1)
    rc1, x1, i1 = _solve(lib, ctx, "dgns_cg_invmass_solve_noalloc", b, mf, x=xb, use_initial_guess=1)
    assert rc0 == 0 and rc1 == 0
    assert i1.iterations == i0.iterations
    assert i1.initial_res == pytest.approx(i0.initial_res, rel=1e-12)
    assert np.max(np.abs(x1 - x0)) <= TOL * np.max(np.abs(x0))


def test_noalloc_allocates_nothing():
    """With the library's next device allocation armed to fail, the call
    still succeeds and the count of live library allocations is unchanged
    (the context is created before the hook is armed)."""
    build_lib()
    from paper_1802_01439_gb300 import _lib
    lib = _lib.load()
    ctx = context((2, 3, 2), 3, mg_precision=0, nu=1.0 / 1600)
    b = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, 3 * ctx.n_u)).cuda()
    _solve(lib, ctx, "dgns_cg_invmass_solve_noalloc", b, 100.0)   # first call: symbol lookup
    live = lib.dgns_debug_live_allocations()
    assert lib.dgns_debug_fail_alloc(1) == 0
    try:
        for _ in range(2):
            rc, x, info = _solve(lib, ctx, "dgns_cg_invmass_solve_noalloc", b, 100.0)
            assert rc == 0 and info.rel_res <= 1e-12
        assert lib.dgns_debug_live_allocations() == live
    finally:
        lib.dgns_debug_fail_alloc(0)


def test_noalloc_rejects_overlap_and_clears_stale_errors():
    build_lib()
    from paper_1802_01439_gb300 import _lib
    lib = _lib.load()
    ctx = context((2, 2, 2), 2, mg_precision=0)
    n = 3 * ctx.n_u
    buf = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    prm = ctx.solve_params()
    rc = lib.dgns_cg_invmass_solve_noalloc(ctx.h, ctypes.c_void_p(buf.data_ptr() + 8 * (n // 2)),
                                           ctypes.c_void_p(buf.data_ptr()), ctypes.c_double(1.0),
                                           ctypes.byref(prm), None)
    assert rc == _lib.DGNS_ERR_ALIAS and b"overlaps" in lib.dgns_last_error()
    b = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, n)).cuda()
    rc, _, _ = _solve(lib, ctx, "dgns_cg_invmass_solve_noalloc", b, 10.0)
    assert rc == 0 and lib.dgns_last_error() == b""


def test_noalloc_rejects_oversized_and_host_input():
    build_lib()
    from paper_1802_01439_gb300 import _lib
    lib = _lib.load()
    big = context((16, 16, 16), 4, mg_precision=0)        # 3 * 512000 entries > 524288
    b = torch.zeros(3 * big.n_u, dtype=torch.float64, device="cuda")
    rc, _, _ = _solve(lib, big, "dgns_cg_invmass_solve_noalloc", b, 1.0)
    assert rc == _lib.DGNS_ERR_INVALID_ARG
    assert b"scratch" in lib.dgns_last_error()
    small = context((2, 2, 2), 2, mg_precision=0)
    bh = torch.zeros(3 * small.n_u, dtype=torch.float64)
    xh = torch.zeros_like(bh)
    prm = small.solve_params()
    rc = lib.dgns_cg_invmass_solve_noalloc(small.h, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(bh.data_ptr()),
                                           ctypes.c_double(1.0), ctypes.byref(prm), None)
    assert rc == _lib.DGNS_ERR_INVALID_ARG
