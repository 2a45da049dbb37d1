"""Oracle: plain FP64 CPU reference of the isogeometric Bratu path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  It shares no code with
the CUDA library (``paper_1305_4452_gb300``) and never imports it.
"""
from .oracle import *  # noqa: F401,F403
