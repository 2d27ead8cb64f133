"""FP64 CPU oracle of the energy-stable FAS multigrid time step.

TEST INFRASTRUCTURE ONLY: ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` are the only importers.  It shares
no code with the CUDA library and never imports it.
"""
from . import scheme, newton  # noqa: F401
