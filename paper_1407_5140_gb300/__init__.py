"""GB300-native replica-exchange Wang-Landau sampling (arXiv:1407.5140).

The sampling runs in the sm_103a CUDA library ``_build/librewl.so`` behind the C
ABI ``include/rewl.h``; ``rewl`` is its Python binding.
"""
from . import rewl  # noqa: F401
from .rewl import ISING, POTTS, Rewl, RewlError, instance  # noqa: F401
