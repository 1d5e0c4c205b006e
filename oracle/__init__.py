"""Test infrastructure: the plain FP64 CPU oracle of the SCMF Monte Carlo step.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package.  The product path never does.
"""
from .oracle import Oracle, OrcDesc, build_oracle, library_path  # noqa: F401
