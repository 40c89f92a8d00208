"""B300-native mixed-state rPIE with Adam position refinement.

The compute path is the C-ABI library ``libpty.so`` (hand-written sm_103a
CUDA, declared in ``include/pty.h``); ``pty`` is its thin ctypes binding.
"""
