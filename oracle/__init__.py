"""FP64 CPU oracle for the tree gravity and collision path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and
the two share no code.  The arithmetic lives in ``rb_oracle.c`` (plain C,
compiled with ``-ffp-contract=off``); this module only marshals numpy arrays.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, load, Params  # noqa: F401
