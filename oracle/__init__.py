"""CPU FP64 oracle for the Lidar surface-segmentation path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (``paper_2005_02704_gb300``) never imports it and has no CPU
fallback.

``lsg_oracle.c`` is a plain, slow, obviously correct FP64 C implementation of
what Mukherjee et al. (PReMI 2019, Sec. 2 and Algorithm 1) define; ``oracle.py``
loads it through ctypes.  It shares no code with the CUDA path.

Parity status: every function is pinned by tests against closed forms, brute
force, the paper's literal Algorithm 1 and invariants, except the end-to-end
segmentation accuracy of the paper's Table 2, which needs the paper's dataset
("parity unpinned" for that table only).
"""
from .oracle import *  # noqa: F401,F403
