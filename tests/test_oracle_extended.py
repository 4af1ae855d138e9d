"""Pins of the oracle's extended-precision path (np.longdouble: 64-bit
significand on x86, binary128 on arm64), which referees the FP64 results of
the convective term where its weak form cancels (Sec. 3.2, c_h with the
over-integration rule): the same discrete operator, every table and product
in the wider precision.

  rules       Gauss rules exact for x^m, m <= 2n-1, to the extended unit
              roundoff, with the closed-form remainder at m = 2n; LGL nodes
              equal their closed forms
              (k = 3, 4) and are roots of P_k'; Lagrange cardinality
  convective  agrees with the FP64 oracle within FP64 rounding of the summed
              terms (and is not the FP64 result); conserves to the extended
              roundoff; the cell-restricted evaluation equals the full one
"""
import numpy as np
import pytest

from oracle import dg, rules
from paper_1802_01439_gb300 import inputs

LD = np.longdouble
EPS = float(np.finfo(LD).eps)

pytestmark = pytest.mark.skipif(EPS >= 1e-18, reason="np.longdouble is no wider than double here")


@pytest.mark.parametrize("n", [2, 5, 12, 18])
def test_extended_gauss_exactness(n):
    x, w = rules.gauss(n, LD)
    assert x.dtype == np.dtype(LD) and w.dtype == np.dtype(LD)
    assert abs(float(w.sum() - 1)) <= 8 * EPS
    for m in range(2 * n):
        exact = LD(1) / (m + 1)
        assert abs(float((w * x ** m).sum() / exact - 1)) <= 64 * n * EPS, m
    # x^2n: the Gauss error on [0, 1] is exactly (n!)^4 / ((2n+1) ((2n)!)^2)
    # (the remainder term f^(2n)(xi) (n!)^4 / ((2n+1) ((2n)!)^3) on [0, 1],
    # with f^(2n) = (2n)! constant)
    from math import factorial
    m = 2 * n
    err = LD(1) / (m + 1) - (w * x ** m).sum()
    closed = LD(factorial(n) ** 4) / LD((2 * n + 1) * factorial(2 * n) ** 2)
    assert abs(float(err - closed)) <= 64 * n * EPS / (m + 1)


def test_extended_lgl_closed_forms():
    s5, s37 = np.sqrt(LD(5)), np.sqrt(LD(3) / LD(7))
    ref = {3: [LD(0), (1 - 1 / s5) / 2, (1 + 1 / s5) / 2, LD(1)],
           4: [LD(0), (1 - s37) / 2, LD(1) / 2, (1 + s37) / 2, LD(1)]}
    for k, r in ref.items():
        x = rules.lgl_nodes(k, LD)
        assert np.max(np.abs(x - np.array(r, dtype=LD))) <= 4 * EPS


@pytest.mark.parametrize("k", [5, 7, 9, 11])
def test_extended_lgl_roots_of_dPk(k):
    x = rules.lgl_nodes(k, LD)
    _, dp = rules.legendre(k, 2 * x[1:-1] - 1)
    # |P_k'| near its roots grows like k^2 per unit of x; the residual is at
    # the extended roundoff, far below what FP64 nodes leave
    assert np.max(np.abs(dp)) <= 1e3 * k ** 2 * EPS
    x64 = rules.lgl_nodes(k)
    _, dp64 = rules.legendre(k, 2 * np.asarray(x64[1:-1], dtype=LD) - 1)
    assert np.max(np.abs(dp64)) > 10 * np.max(np.abs(dp))


def test_extended_lagrange_partition_of_unity():
    nodes = rules.lgl_nodes(7, LD)
    g, _ = rules.gauss(12, LD)
    V, D = rules.lagrange(nodes, g, LD)
    assert np.max(np.abs(V.sum(axis=1) - 1)) <= 256 * EPS
    assert np.max(np.abs(D.sum(axis=1))) <= 4096 * EPS
    C, _ = rules.lagrange(nodes, nodes, LD)
    assert np.max(np.abs(C - np.eye(8, dtype=LD))) <= 64 * EPS


def _fields(m, k):
    return inputs.taylor_green(m.n, m.lo, m.hi, rules.lgl_nodes(k), noise=1e-3, seed=0)


@pytest.mark.parametrize("n,k", [((3, 3, 3), 3), ((2, 3, 2), 5), ((3, 2, 2), 7)])
def test_extended_convective_agrees_with_fp64(n, k):
    m = dg.Mesh(n)
    me = dg.Mesh(n, dtype=LD)
    s, se = dg.Space(m, k), dg.Space(me, k)
    U = _fields(m, k)
    C = dg.Convective(s)
    y, mag = C.apply(U), C.magnitude(U)
    ye = dg.Convective(se).apply(U)
    assert ye.dtype == np.dtype(LD)
    diff = np.abs(y - ye)
    assert np.max(diff) <= 1e-14 * np.max(mag)        # FP64 rounding of the summed terms
    assert np.max(diff) > 0                           # and it is not the FP64 evaluation


@pytest.mark.parametrize("k", [2, 4])
def test_extended_convective_conserves(k):
    me = dg.Mesh((2, 3, 2), dtype=LD)
    se = dg.Space(me, k)
    U = np.random.default_rng(3).uniform(-1, 1, (3, me.E, se.ndofs_cell))
    Ce = dg.Convective(se)
    Y = Ce.apply(U)
    scale = float(np.max(np.abs(Y)))
    assert float(np.max(np.abs(Y.sum(axis=(1, 2))))) <= 64 * EPS * scale * Y[0].size


@pytest.mark.parametrize("dtype", [np.float64, LD])
def test_convective_restricted_to_cells(dtype):
    m = dg.Mesh((3, 2, 3), dtype=dtype)
    s = dg.Space(m, 3)
    U = np.random.default_rng(5).uniform(-1, 1, (3, m.E, s.ndofs_cell))
    C = dg.Convective(s)
    full = C.apply(U)
    sel = [0, 7, 17]
    part = C.apply(U, cells=sel)
    tol = 1e-14 if dtype is np.float64 else 64 * EPS
    assert np.max(np.abs(part[:, sel] - full[:, sel])) <= tol * np.max(np.abs(full))
    rest = [e for e in range(m.E) if e not in sel]
    assert np.max(np.abs(part[:, rest])) == 0
