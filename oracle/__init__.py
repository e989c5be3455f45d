"""CPU oracle (FP64) for the parallel-in-time multilevel Krylov method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.
It shares no code with the CUDA implementation.
"""
from .mk_oracle import *  # noqa: F401,F403
