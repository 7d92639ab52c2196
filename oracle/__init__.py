"""CPU oracle for the fJOFC hot path (float64, dense, slow, obviously correct).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.  See ``fjofc_oracle`` for
what each function computes and which passage of the paper it follows, and
``mlp_oracle`` for the warm-start network's float64 reference.
"""
from .fjofc_oracle import *  # noqa: F401,F403
