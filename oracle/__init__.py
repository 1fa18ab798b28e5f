"""Plain FP64 CPU oracle for the generalized vec trick (GVT) path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it, and it never imports the product package.
"""
from .oracle import *  # noqa: F401,F403
