"""B300-native SCMF Monte Carlo step (libsoma) and its Python binding.

The package holds the CUDA sources (``csrc/``), the in-tree build
(``build.py`` -> ``libsoma.so``), the ctypes binding of the C ABI in
``include/soma.h`` (``soma.py``) and the workload definitions
(``workloads.py``).
"""
from . import soma  # noqa: F401
from .soma import Handle, System  # noqa: F401
