"""FP64 CPU oracle of the L-ACE exchange hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1801_09263_gb300``; the two meet only on the seeded
inputs produced by ``synth``.
"""
from .lace_oracle import *  # noqa: F401,F403
from .lace_oracle import __all__  # noqa: F401
