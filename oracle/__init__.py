"""Plain CPU oracle for the QAOA hot path (arXiv 2309.04841).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls anything here.  See ``oracle/oracle.c`` for the definitions
each routine follows.
"""
from .oracle import *  # noqa: F401,F403
