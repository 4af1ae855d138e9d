"""Helpers shared by the GPU parity tests: build the library, create contexts,
move seeded inputs to the device and measure the relative max-norm error."""
import numpy as np
import torch

from oracle import rules
from paper_1802_01439_gb300 import inputs

PI = np.pi


def build_lib():
    from paper_1802_01439_gb300 import build
    build.build()


def context(n, k, kp=-1, **kw):
    from paper_1802_01439_gb300 import Context
    return Context(n, k, degree_p=kp, **kw)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda().contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().double().numpy()


def rel_err(y, ref, scale=None):
    """Relative max-norm error ||y - ref||_inf / ||ref||_inf (or / scale)."""
    y = np.asarray(y).ravel()
    ref = np.asarray(ref).ravel()
    s = scale if scale is not None else np.max(np.abs(ref))
    return float(np.max(np.abs(y - ref)) / s)


def random_field(space, ncomp, seed):
    shape = (ncomp, space.mesh.E, space.ndofs_cell) if ncomp > 1 else (space.mesh.E, space.ndofs_cell)
    return inputs.uniform(seed, int(np.prod(shape))).reshape(shape)


def tgv_field(space, noise, seed):
    m = space.mesh
    return inputs.taylor_green(m.n, m.lo, m.hi, rules.lgl_nodes(space.k), noise=noise, seed=seed)
