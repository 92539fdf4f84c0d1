"""GB300-native vacuum-arc PIC-MCC step (Koitermaa et al., arXiv:2402.08404).

The compute path is the C-ABI library ``libpic.so`` (hand-written CUDA for sm_103a) declared
in ``include/pic.h``; ``paper_2402_08404_gb300.pic`` is its thin ctypes binding.  Importing
this package loads nothing; ``synth`` holds the seeded workload generators.
"""
__all__ = ["pic", "synth"]
