"""FP64 CPU oracle of the hydro right-hand side (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.  See ``oct_oracle.c`` for the method and the
readings of the paper it fixes.
"""
from .oracle import *  # noqa: F401,F403
