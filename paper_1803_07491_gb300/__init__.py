"""GB300-native analytic bond-order potential (BOP) hot path.

Moments of an orthogonal Slater-Koster tight-binding Hamiltonian, the
recursion, the constant-terminator expansion of the local DOS, the Fermi
level with local-charge-neutrality / Stoner self-consistency, the bond
energy and its exact gradient (forces, virial), after the BOPfox paper
(arXiv:1803.07491).  Every step runs in the CUDA kernels of
``libbopgb.so``; ``paper_1803_07491_gb300.bop`` is the thin ctypes binding.

Importing this package loads nothing; the library is loaded on first use
and a missing library is an error, never a fallback.
"""
