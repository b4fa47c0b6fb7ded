"""B300-native lattice Landau-de Gennes force + FIRE minimiser.

``lqmin`` is the thin ctypes binding over the C-ABI library ``liblqmin.so``
(built from ``csrc/`` for sm_103a); ``synth`` produces seeded inputs.
Importing the package does not load the CUDA library; the first call into
``lqmin`` does, and fails loudly if it has not been built.
"""
__all__ = ["lqmin", "synth"]
