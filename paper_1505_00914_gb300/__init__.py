"""GB300-native (sm_103a) integer convex-hull preconditioner.

Cadenas & Megson's Algorithm 1 reduces n integer points in [1,p]^2 to one
(min y, max y) pair per x column; the valid columns form x-ordered lower and
upper chains (Lemma 1) on which a monotone-chain hull runs with no sort.  Every
step is a hand-written CUDA kernel in ``libch.so`` behind the C ABI declared in
``include/ch.h``; ``paper_1505_00914_gb300.ch`` is the thin ctypes binding.

Importing the package loads nothing; ``paper_1505_00914_gb300.ch`` loads the
CUDA library on first use and raises if it is missing.
"""

__all__ = ["ch", "synth"]
