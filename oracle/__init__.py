"""CPU FP64 oracle for the Taylor–Couette time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this package.  The product path
(``paper_1311_2481_gb300`` and its CUDA library) never imports it and shares no code with
it; both sides only share the seeded input generators in ``paper_1311_2481_gb300.inputs``.
"""
from .tc_oracle import *  # noqa: F401,F403
