"""The C-ABI library builds, loads and exports every entry point that
include/dgns.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_01439_gb300 import _lib, build
    build.build()
    return _lib.load()


def header_functions():
    with open(os.path.join(ROOT, "include", "dgns.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgns_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("dgns_create", "dgns_vmult_laplace", "dgns_vmult_convective",
                     "dgns_vmult_viscous", "dgns_apply_inverse_mass", "dgns_cg_mg_solve"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1802_01439_gb300 import _lib
    for name in header_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding misses " + name


def test_defaults_and_strings(lib):
    from paper_1802_01439_gb300 import _lib
    d = _lib.MeshDesc()
    lib.dgns_default_desc(ctypes.byref(d))
    assert list(d.n_elem) == [4, 4, 4] and d.degree == 3 and d.degree_p == -1
    assert abs(d.hi[0] - 3.141592653589793) < 1e-15 and d.mg_precision == 32
    p = _lib.SolveParams()
    lib.dgns_default_solve_params(ctypes.byref(p))
    assert p.cheb_degree == 5 and p.smoothing_range == 20.0 and p.rel_tol == 1e-10
    for code in range(8):
        assert lib.dgns_status_string(code)


@pytest.mark.parametrize("field,value", [("degree", 0), ("degree", 12), ("degree_p", 13),
                                         ("mg_precision", 16), ("n_q_conv", 7)])
def test_create_rejects_bad_descriptions(lib, field, value):
    from paper_1802_01439_gb300 import _lib
    d = _lib.MeshDesc()
    lib.dgns_default_desc(ctypes.byref(d))
    setattr(d, field, value)
    h = ctypes.c_void_p(1)
    rc = lib.dgns_create(ctypes.byref(d), None, ctypes.byref(h))
    assert rc in (_lib.DGNS_ERR_INVALID_ARG, _lib.DGNS_ERR_UNSUPPORTED)
    assert h.value is None
    assert lib.dgns_last_error()


def test_create_rejects_bad_mesh(lib):
    from paper_1802_01439_gb300 import _lib
    d = _lib.MeshDesc()
    lib.dgns_default_desc(ctypes.byref(d))
    d.n_elem[1] = 0
    h = ctypes.c_void_p()
    assert lib.dgns_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.DGNS_ERR_INVALID_ARG
    d.n_elem[1] = 4
    d.hi[2] = d.lo[2]
    assert lib.dgns_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.DGNS_ERR_INVALID_ARG


def test_null_context_is_rejected(lib):
    from paper_1802_01439_gb300 import _lib
    assert lib.dgns_vmult_laplace(None, None, None, 0) == _lib.DGNS_ERR_INVALID_ARG
    assert lib.dgns_cg_mg_solve(None, None, None, None, None) == _lib.DGNS_ERR_INVALID_ARG


def test_create_rejects_oversized_mesh(lib):
    """3 x cells >= 2^31 exceeds the 32-bit cell indexing of the kernels: the
    description is rejected (unsupported) before any allocation."""
    from paper_1802_01439_gb300 import _lib
    d = _lib.MeshDesc()
    lib.dgns_default_desc(ctypes.byref(d))
    d.n_elem[0] = d.n_elem[1] = d.n_elem[2] = 900     # 7.29e8 cells, 3 x = 2.19e9
    h = ctypes.c_void_p()
    assert lib.dgns_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.DGNS_ERR_UNSUPPORTED
    assert h.value is None and b"2^31" in lib.dgns_last_error()


def test_null_arguments_of_new_entry_points(lib):
    from paper_1802_01439_gb300 import _lib
    E = _lib.DGNS_ERR_INVALID_ARG
    n = ctypes.c_longlong()
    assert lib.dgns_convective_face_size(None, ctypes.byref(n)) == E
    assert lib.dgns_convective_faces(None, None, None) == E
    assert lib.dgns_convective_cells(None, None, None, None) == E
    assert lib.dgns_vmult_projection(None, None, None, None, None) == E
    assert lib.dgns_cg_projection_solve(None, None, None, None, None, None, None) == E
    assert lib.dgns_penalty_parameters(None, None, 1.0, 1.0, 1.0, None, None) == E


def test_solve_params_layout(lib):
    """The binding's SolveParams mirrors the header (the default fills every
    field, the initial-guess switch included)."""
    from paper_1802_01439_gb300 import _lib
    p = _lib.SolveParams()
    p.use_initial_guess = 7
    lib.dgns_default_solve_params(ctypes.byref(p))
    assert p.use_initial_guess == 0 and p.project_mean == 1 and p.abs_tol == 0.0


def test_allocation_failure_hook_arguments(lib):
    """The failure-path hooks need no device: n < 0 is rejected, 0 disarms,
    and nothing is allocated before any context exists."""
    from paper_1802_01439_gb300 import _lib
    assert lib.dgns_debug_fail_alloc(-1) == _lib.DGNS_ERR_INVALID_ARG
    assert lib.dgns_debug_fail_alloc(3) == 0
    assert lib.dgns_debug_fail_alloc(0) == 0
    assert lib.dgns_debug_live_allocations() == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libdgns.so, loading the library and creating
    a context raise instead of computing anything."""
    from paper_1802_01439_gb300 import Context, _lib
    missing = str(tmp_path / "libdgns.so")
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(missing)
    monkeypatch.setattr(_lib, "LIB_PATH", missing)
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        Context(2, 2)
