"""B300-native hot path of Gerbil's two-phase k-mer counter (arXiv 1607.06618).

The CUDA library ``libgerbil.so`` (built from ``csrc/``) holds every step of the path; the
``gerbil`` module is a thin ctypes binding with the C-ABI's names.  ``synth`` draws seeded
synthetic read sets.
"""
