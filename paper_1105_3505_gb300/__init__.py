"""GB300-native lattice fast multipole method (Gillman & Martinsson, arXiv 1105.3505).

Evaluates u(m) = sum_n phi(m - n) f(n) on Z^2 (eq. 1.7), phi the fundamental
solution of the 5-point discrete Laplacian, with the lattice FMM of Sec. 8 on
one GPU.  The CUDA library (``liblfmm.so``, C ABI in include/lfmm.h) does all
the work; ``lfmm`` is its thin ctypes binding.  ``workloads`` holds the seeded
synthetic inputs.  Importing the package does not load the CUDA library;
``paper_1105_3505_gb300.lfmm`` loads it on first use and raises if it is absent.
"""
__all__ = ["lfmm", "workloads"]
