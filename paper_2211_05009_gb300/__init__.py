"""GB300 (sm_103a) D2Q9 lattice Boltzmann lid-driven cavity library.

Implements the time step of Xiang & Shi (arXiv 2211.05009) -- BGK collision and streaming
(Eq. 1-3), non-equilibrium-extrapolation walls and moving lid (Sec. 2.2), the Eq. 6 residual and
the stream-function post-processing of Tables 1-2 -- as hand-written CUDA behind the C ABI of
``include/lbm.h``.  ``binding`` mirrors the C entry points one to one; ``Cavity`` wraps a context.
"""
from .binding import LBMError, DTYPES, library  # noqa: F401

__all__ = ["LBMError", "DTYPES", "library", "Cavity", "build"]


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)


def __getattr__(name):
    if name == "Cavity":
        from .cavity import Cavity
        return Cavity
    raise AttributeError(name)
