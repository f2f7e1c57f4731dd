"""GB300-native (sm_103a) restarted PDHG for discrete optimal transport
(PDOT, arXiv 2407.19689).

- ``pdot``: ctypes binding of the C ABI (``include/pdot.h``) and a torch-tensor
  ``Solver`` wrapper.  The solver runs entirely in ``libpdot.so``.
- ``instances``: seeded synthetic OT workloads (inputs only).
- ``serve``: Poisson request driver for the continuous-batching engine.
"""
from ._build import build  # noqa: F401

__all__ = ["build"]
