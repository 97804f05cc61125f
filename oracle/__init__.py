"""FP64 CPU oracle for the MPS two-qubit-gate path -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct reference that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg and ``--impl reference`` arm may import it.  The library in
``paper_2601_04422_gb300`` never imports it and shares no code with it.

Modules
-------
mps    -- the MPS simulator (Eq. 2 state, Eq. 3 one-qubit gates, the merge /
          gate / SVD / absorb two-qubit update, layers, amplitudes, Pauli
          expectations, overlaps, canonical forms, perfect sampling).
dense  -- a direct state-vector simulator (the full contraction of Eq. 1), used
          to pin ``mps`` on small qubit counts where nothing is truncated.
grad   -- the reverse-mode gradient of an energy through the layered simulation
          (the exact derivative of the truncated updates), pinned by finite
          differences of the dense and of the truncated energies.

Every function is complex128 / float64, except ``mps.apply_2q_single_precision``,
which rounds the stored sites to complex64 and contracts in complex64 around an
exact FP64 SVD: the precision floor that no complex64 path can go below.  The
singular value decomposition step calls LAPACK through ``numpy.linalg.svd`` (a
library primitive).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
the dense simulator, closed forms (GHZ, QFT of a basis state), invariants or
designed spectra -- except the truncated regime at a degenerate cut, where the
kept subspace is not unique ("parity unpinned": only singular values and
discarded weights are compared there).
"""
from . import dense, grad, mps  # noqa: F401
