"""GB300 (sm_103a) implementation of the IUGKP steady-state phonon BTE sweep
(Liu, Yang, Zhang, Ji, Xu, arXiv 2506.09465): a C-ABI CUDA library (libiugkp.so, see
include/iugkp.h) and this thin Python binding. The library is loaded on first use and
there is no CPU fallback."""
from ._lib import IugkpError, load  # noqa: F401


def __getattr__(name):
    if name in ("Solver", "GridSpec", "IugkpSteady"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
