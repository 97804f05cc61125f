"""Dense state-vector simulator: the direct contraction of the circuit network (Eq. 1).

The paper rejects this method for large widths because its cost is exponential in
the number of qubits (Sec. II.A), which is exactly why it is a good *pin* for the
MPS oracle at <= 12 qubits: it shares no step with the MPS update (no merge, no SVD,
no truncation), so a dropped term, a wrong index or a transposed operand in the MPS
code shows up as an amplitude mismatch.

Qubit 0 is the most significant bit of the dense index (axis 0 of the
``(2,)*n`` view).  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .mps import PAULI


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    """Contract a rank-2 gate tensor with leg q of the rank-n state tensor (Eq. 1, U^(1))."""
    t = psi.reshape((2,) * n)
    t = np.tensordot(u, t, axes=([1], [q]))      # new axis 0 = output leg
    t = np.moveaxis(t, 0, q)
    return t.reshape(-1)


def apply_2q(psi: np.ndarray, n: int, q: int, g: np.ndarray) -> np.ndarray:
    """Contract a rank-4 gate tensor with legs (q, q+1) (Eq. 1, U^(2)).

    ``g`` is 4x4 with basis index 2*b_q + b_{q+1}; as a tensor G[a, b, c, d] it maps
    input legs (c, d) to output legs (a, b).
    """
    t = psi.reshape((2,) * n)
    G = g.reshape(2, 2, 2, 2)
    t = np.tensordot(G, t, axes=([2, 3], [q, q + 1]))   # axes 0,1 = outputs
    t = np.moveaxis(t, [0, 1], [q, q + 1])
    return t.reshape(-1)


def apply_2q_any(psi: np.ndarray, n: int, qa: int, qb: int, g: np.ndarray) -> np.ndarray:
    """Contract a rank-4 gate tensor with legs (qa, qb) of the state, any two distinct
    qubits in either order (Eq. 1, U^(2) on non-adjacent legs); ``g`` has basis index
    2*b_qa + b_qb."""
    t = psi.reshape((2,) * n)
    G = g.reshape(2, 2, 2, 2)
    t = np.tensordot(G, t, axes=([2, 3], [qa, qb]))
    t = np.moveaxis(t, [0, 1], [qa, qb])
    return t.reshape(-1)


def run_ops(n: int, ops) -> np.ndarray:
    """A gate list in program order; (qa, qb, matrix) with qb None or < 0 for one qubit."""
    psi = zero_state(n)
    for qa, qb, g in ops:
        g = np.asarray(g, dtype=np.complex128)
        if qb is None or qb < 0:
            psi = apply_1q(psi, n, int(qa), g)
        else:
            psi = apply_2q_any(psi, n, int(qa), int(qb), g)
    return psi


def run_circuit(circuit) -> np.ndarray:
    """Apply every layer: the layer's one-qubit gates first, then its two-qubit gates."""
    n = circuit.n_qubits
    psi = zero_state(n)
    for layer in circuit.layers:
        if layer.u1 is not None:
            for q in range(n):
                psi = apply_1q(psi, n, q, layer.u1[q])
        for q, g in zip(layer.pairs, layer.g4):
            psi = apply_2q(psi, n, int(q), g)
    return psi


def amplitude(psi: np.ndarray, n: int, bits) -> complex:
    idx = 0
    for b in bits:
        idx = (idx << 1) | int(b)
    return complex(psi[idx])


def expect_pauli(psi: np.ndarray, n: int, pstring: str) -> complex:
    """<psi| P_0 (x) P_1 (x) ... |psi> by applying each Pauli to a copy of the vector."""
    phi = psi.copy()
    for q, c in enumerate(pstring):
        if c != "I":
            phi = apply_1q(phi, n, q, PAULI[c])
    return complex(np.vdot(psi, phi))
