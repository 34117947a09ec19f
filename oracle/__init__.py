"""CPU oracle of the Virtual Transmission Method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The CUDA library never uses it.
"""
from .vtm_oracle import *  # noqa: F401,F403
