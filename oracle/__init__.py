"""CPU oracle for the VG-rtTDDFTB propagation path (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package; the library never does.
"""
from .vgtb_oracle import *  # noqa: F401,F403
from . import vgtb_oracle  # noqa: F401
from . import crank_nicolson  # noqa: F401
from .crank_nicolson import propagate_cn  # noqa: F401
