"""GB300 (sm_103a) implementation of the MACE hot path of multi-slice fusion
(arXiv 2008.01567): a C-ABI CUDA library (csrc/, include/msf.h), its thin ctypes
binding (msf.py), the in-tree build (build.py) and the seeded input generators
(synth.py)."""
from . import synth  # noqa: F401
