"""FP64 CPU oracle for u-series electrostatics (arXiv:1911.01377).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users.  It shares no code with the
GPU library in ``paper_1911_01377_gb300``; the two meet only at the seeded
input generators.

Parity pinned: every function here is checked by ``tests/test_oracle_*.py``
against values the paper prints (Tables 1-2, the M_b bounds, the Eq. 33
worked example), closed forms (the NaCl Madelung constant), an independent
classic Ewald sum, a real-space image sum and finite differences.
"""
from .oracle import *  # noqa: F401,F403
from . import series  # noqa: F401
