"""GB300 (sm_103a) solve phase of an AMG-preconditioned Krylov solver for
sparse systems A X = B with m right-hand sides.

* ``problems``: seeded synthetic test systems (Poisson 7/27-point, RHS blocks).
* ``binding``: ctypes binding of the C ABI (``include/xamg_gpu.h``) of the
  CUDA library built in-tree by ``build``.
"""
from . import problems  # noqa: F401

__all__ = ["problems", "build", "binding"]
