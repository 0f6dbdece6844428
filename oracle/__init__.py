"""FP64 CPU oracle for the fast 3D super-resolution method (arXiv:2010.15491).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The CUDA library (paper_2010_15491_gb300) never
imports it and shares no code with it.
"""
from . import sr3d_oracle, dense  # noqa: F401
from .sr3d_oracle import *  # noqa: F401,F403
