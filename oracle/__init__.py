"""CPU FP64 oracle -- test infrastructure only.

Importable only from ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product library never imports it.
"""
from .oracle import *  # noqa: F401,F403
