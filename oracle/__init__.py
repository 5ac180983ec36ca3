"""CPU oracle for the SP2 / SP2ACC density-matrix expansion (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline
leg and ``--impl reference``) may import this package.  The CUDA library never
does, and the two share no code: the oracle restates the paper's steps in plain
numpy FP64 so that a reader can check them by eye.
"""
from .sp2_oracle import *  # noqa: F401,F403
