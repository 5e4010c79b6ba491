"""FP64 CPU oracle of the explicit EBE enthalpy step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

``parity unpinned`` does not apply to any function here: every function is
pinned by the ``tests/test_oracle_*.py`` suite (closed forms, an independent
barycentric stiffness, patch test, lumping sums, T(E) round trips, energy
conservation, erfc/erf slabs, the Neumann Stefan problem and the eigenvalue
stability limit).

``oracle.surrogate`` is the plain CPU definition of the learned mesh
surrogate (features, forward and backward pass with the kernels' bf16
rounding points, Adam), pinned by ``tests/test_oracle_surrogate.py``
(the FE oracle's explicit residual, a patch test, a brute-force forward,
finite differences and torch's Adam).
"""
from .oracle import (OracleProblem, build, E_from_T, T_from_E, liquid_fraction,
                     tet_matrix)

__all__ = ["OracleProblem", "build", "E_from_T", "T_from_E", "liquid_fraction",
           "tet_matrix"]
