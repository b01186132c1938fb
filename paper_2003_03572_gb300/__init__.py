"""GB300-native Saturating Coordinate Descent (SaCD) for sparse nonnegative CP factorisation.

The compute path is the CUDA library ``libsacd.so`` (C-ABI declared in ``include/sacd.h``);
``paper_2003_03572_gb300.sacd`` is its thin ctypes binding. Importing this package does not
load the library; the first call through the binding does, and fails loudly if it is missing.
"""

__all__ = ["sacd", "synth"]
