"""GB300-native PCG for SPD block-tridiagonal systems with the optimal
multi-splitting polynomial preconditioner (arXiv 2503.15269).

The compute path is the CUDA library ``libbt.so`` built from ``csrc/``; this
package only marshals arguments to it (``binding``) and wraps it for autograd.
Importing the package does not load the library; the first call does, and
raises if it is missing.
"""
from . import workloads  # noqa: F401  (pure numpy input generators)

__all__ = ["workloads"]
