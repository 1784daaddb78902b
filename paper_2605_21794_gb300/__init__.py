"""GB300 (sm_103a) implementation of the decorated-particle (Scovel-Weinstein,
k = 2) step for the 1D1V periodic Vlasov-Poisson system.

The compute path is ``_build/libswpic.so`` (CUDA kernels behind the C ABI of
``include/swpic.h``); ``swpic`` is its thin ctypes binding.  Importing this
package does not load the library; the first call into ``swpic`` does, and
fails loudly when the library is missing.
"""
from . import swpic  # noqa: F401

__all__ = ["swpic"]
