"""GB300-native full-range dispersion-encoded ISAM (arXiv 1905.06058).

The CUDA kernels and the C ABI live in ``csrc/`` and build into ``libisam.so``
next to this file; ``isam`` is the thin ctypes binding over that ABI (plans,
A / A^H, solves with their priors, batches as CUDA graphs, the filter, the
direct Eq. 9 reconstruction, autotuning, the allocator hook), ``calib`` wraps
the calibration entry points as torch.autograd.Functions, and ``inputs`` is the
seeded synthetic-workload generator.  Import ``isam`` lazily so that CPU-only
tools can use ``inputs`` without the CUDA library.
"""
