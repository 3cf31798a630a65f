"""GB300 (sm_103a) bit-vectorized octahedron-model SCA: CUDA kernels behind a C ABI.

The compiled library ``libsca.so`` (built by ``build.py``) holds every kernel; ``sca`` is its
ctypes binding.  Importing this package loads nothing; the library is loaded on first use.
"""
from . import build  # noqa: F401
