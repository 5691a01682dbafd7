"""GB300 (sm_103a) off-lattice Boltzmann step for van der Waals fluids.

The compute path is the C-ABI library ``libolb.so`` built from ``csrc/``
(hand-written CUDA for sm_103a); ``olb`` is its thin ctypes binding and
``build`` compiles it in-tree.  ``inputs`` builds seeded synthetic initial
conditions.  Importing ``paper_1702_01690_gb300.olb`` raises if the library
has not been built: there is no CPU fallback.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "olb", "build"]
