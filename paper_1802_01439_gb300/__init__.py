"""GB300-native matrix-free DG operators and solvers for the incompressible
Navier-Stokes dual-splitting scheme of Fehn, Wall & Kronbichler
(arXiv:1802.01439).

The compute path is libdgns (CUDA, sm_103a) behind the C ABI in
include/dgns.h; ``Context`` is its Python binding.  Importing this package
does not load the library; creating a ``Context`` does, and fails loudly when
it is not built.
"""
from ._lib import SPACE_P, SPACE_U, DgnsError  # noqa: F401


def __getattr__(name):
    if name == "Context":
        from .context import Context
        return Context
    raise AttributeError(name)
