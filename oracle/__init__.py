"""Plain FP64 CPU oracle of the analytic-BOP moments path (arXiv:1803.07491).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import this package.  It shares no code with the CUDA path in
``paper_1803_07491_gb300``; both sides only take the seeded inputs made by
``paper_1803_07491_gb300.inputs``.

Parity status of each function is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
from .bop import (  # noqa: F401
    Model, Settings, neighbors, blocks, cluster, moments, moments_adjoint,
    bond_gradient, edge_vectors, sk_block, recursion_coefficients, gershgorin,
    normalised_moments, cheb_p, sigma_from_moments, zeta_sigma, jackson,
    chi_hat, orbital_N_U, dos_at, fermi_bisect, scalar_stage, weights,
    evaluate, moments_nc, moments_nc_adjoint, local_moments, global_weights,
    pauli_vector,
)
