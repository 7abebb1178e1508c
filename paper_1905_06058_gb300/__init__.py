"""GB300-native full-range dispersion-encoded ISAM (arXiv 1905.06058).

The CUDA kernels and the C ABI live in ``csrc/`` and build into ``libisam.so``
next to this file; ``isam`` is the thin ctypes binding over that ABI and
``inputs`` the seeded synthetic-workload generator.  Import ``isam`` lazily so
that CPU-only tools can use ``inputs`` without the CUDA library.
"""
