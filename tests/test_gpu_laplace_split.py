"""The SIPG Laplacian evaluated operator by operator (cell term, face kernel,
face-apply kernel; Sec. 3.2) against the oracle's assembled element and face
matrices, and against the fused kernel, k = 1..11, on meshes with different
cell counts per direction (one of them a single cell, its own neighbour)."""
import numpy as np
import pytest
import torch

from oracle import dg
from tests.gpu_common import build_lib, context, dev, host, random_field, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib()


@pytest.mark.parametrize("n,k", [((3, 2, 4), 1), ((2, 3, 2), 2), ((4, 2, 3), 3), ((1, 3, 2), 4), ((2, 2, 3), 5),
                                 ((2, 1, 2), 7), ((1, 2, 2), 9), ((2, 1, 1), 11)])
@pytest.mark.parametrize("space", [0, 1])
def test_split_laplace_matches_oracle_and_fused(n, k, space):
    ctx = context(n, k, max(k - 1, 1), mg_precision=0)
    kk = k if space == 0 else max(k - 1, 1)
    s = dg.Space(dg.Mesh(n), kk)
    x = random_field(s, 1, 7 + k)
    y = torch.empty(s.size, dtype=torch.float64, device="cuda")
    ctx.vmult_laplace_split(y, dev(x), space)
    ref = dg.Laplace(s).apply(x)
    assert rel_err(host(y), ref) <= 1e-12
    yf = torch.empty_like(y)
    ctx.vmult_laplace(yf, dev(x), space)
    assert rel_err(host(y), host(yf)) <= 1e-13


def test_split_laplace_host_buffers_and_repeat():
    """Host vectors are staged; a second call on the larger space regrows the
    face buffer; results repeat exactly."""
    ctx = context((3, 2, 2), 4, 2, mg_precision=0)
    for space, kk in ((1, 2), (0, 4), (1, 2)):
        s = dg.Space(dg.Mesh((3, 2, 2)), kk)
        x = random_field(s, 1, 3)
        xt = torch.from_numpy(np.ascontiguousarray(x.ravel()))
        y = torch.empty(s.size, dtype=torch.float64)
        ctx.vmult_laplace_split(y, xt, space)
        assert rel_err(y.numpy(), dg.Laplace(s).apply(x)) <= 1e-12
        y2 = torch.empty(s.size, dtype=torch.float64)
        ctx.vmult_laplace_split(y2, xt, space)
        assert torch.equal(y, y2)


def test_split_laplace_rejects_bad_arguments():
    from paper_1802_01439_gb300 import DgnsError
    ctx = context((2, 2, 2), 3, 2, mg_precision=0)
    n = ctx.n_p
    x = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    rc = ctx.lib.dgns_vmult_laplace_split(ctx.h, x.data_ptr(), x.data_ptr() + 8, 1)
    assert rc != 0                                    # dst overlaps src
    rc = ctx.lib.dgns_vmult_laplace_split(ctx.h, x.data_ptr(), x[n:].data_ptr(), 5)
    assert rc != 0                                    # no such space
    with pytest.raises(DgnsError):
        ctx.vmult_laplace_split(torch.empty(n, dtype=torch.float64, device="cuda"), x[:n] * 1.0, 5)
