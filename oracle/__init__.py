"""FP64 CPU oracle of the FITrig trigger path.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; never by the CUDA library or its binding.
"""
from . import fitrig_oracle  # noqa: F401
