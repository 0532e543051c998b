"""GB300 (sm_103a) solver for the fractional Laplacian with extended
Dirichlet conditions (Minden & Ying, arXiv:1802.03770).

* ``api.Plan``      -- operator plan: apply, preconditioner, solves, time steps
* ``_lib``          -- ctypes binding of include/fraclap.h (libfraclap.so)
* ``inputs``        -- seeded synthetic inputs
* ``build``         -- builds libfraclap.so in-tree for sm_103a
"""

from . import inputs  # noqa: F401

__all__ = ["inputs", "Plan", "load"]


def load():
    from . import _lib
    return _lib.load()


def __getattr__(name):
    if name == "Plan":
        from .api import Plan
        return Plan
    raise AttributeError(name)
