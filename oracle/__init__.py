"""FP64 CPU oracle of the patch-hashing zoom (test infrastructure only).

This package is test infrastructure.  Only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library and imports nothing from it; both sides receive the same
seeded inputs from ``synth_inputs``.
"""
from .zoom_oracle import *  # noqa: F401,F403
