"""Seeded synthetic circuits and site tensors.

Everything here is *input*: gate matrices, which qubits they act on, and random
tensors.  Both the CUDA path and the FP64 oracle consume the same arrays, so a
parity test compares the two implementations on identical data.

Conventions (fixed once, used everywhere):

* qubit 0 is the leftmost MPS site and the most significant bit of a dense index;
* a two-qubit gate on the adjacent pair (q, q+1) is a 4x4 complex matrix whose
  basis index is ``2*b_q + b_{q+1}`` (row = output, column = input);
* a one-qubit gate is a 2x2 matrix acting on the physical leg (Eq. 3);
* a layer is a set of two-qubit gates on disjoint adjacent pairs (Sec. IV.B,
  "Parallelizing the TAMM Backend", layerization) plus optional one-qubit
  gates on every qubit that act *before* the two-qubit gates of the layer.

Haar-random unitaries follow Mezzadri, "How to generate random matrices from the
classical compact groups" (Notices AMS 54, 2007): QR of a complex Ginibre matrix
with the phases of R's diagonal moved into Q.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Layer", "Circuit",
    "haar_unitary", "haar_su4", "gate_h", "gate_x", "gate_y", "gate_z",
    "gate_rx", "gate_ry", "gate_rz", "gate_cx", "gate_cz", "gate_swap",
    "gate_rzz", "gate_cp", "PAULI",
    "brickwork_su4", "brickwork_u2_su4", "gateset_circuit", "hea_circuit",
    "ghz_circuit", "qft_nn_circuit", "batch_circuits", "random_sites",
    "random_bitstrings", "config_c1", "config_c2", "config_c3", "nonlocal_ops",
]


# --------------------------------------------------------------------------
# data containers


@dataclass
class Layer:
    """One layer: two-qubit gates on disjoint pairs (q, q+1), optional 1q gates first."""

    pairs: np.ndarray                      # int32 [n2]  left qubit of each pair
    g4: np.ndarray                         # complex128 [n2, 4, 4]
    u1: Optional[np.ndarray] = None        # complex128 [n_qubits, 2, 2] or None

    def __post_init__(self):
        self.pairs = np.ascontiguousarray(self.pairs, dtype=np.int32).reshape(-1)
        self.g4 = np.ascontiguousarray(self.g4, dtype=np.complex128).reshape(-1, 4, 4)
        assert self.g4.shape[0] == self.pairs.shape[0]
        if self.u1 is not None:
            self.u1 = np.ascontiguousarray(self.u1, dtype=np.complex128)

    @property
    def n2(self) -> int:
        return int(self.pairs.shape[0])


@dataclass
class Circuit:
    n_qubits: int
    layers: List[Layer] = field(default_factory=list)
    meta: dict = field(default_factory=dict)

    @property
    def n_2q(self) -> int:
        return sum(l.n2 for l in self.layers)


# --------------------------------------------------------------------------
# gate matrices


PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def gate_h() -> np.ndarray:
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def gate_x() -> np.ndarray:
    return PAULI["X"].copy()


def gate_y() -> np.ndarray:
    return PAULI["Y"].copy()


def gate_z() -> np.ndarray:
    return PAULI["Z"].copy()


def gate_rx(t: float) -> np.ndarray:
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def gate_ry(t: float) -> np.ndarray:
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def gate_rz(t: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * t), np.exp(0.5j * t)]).astype(np.complex128)


def gate_cx() -> np.ndarray:
    """CNOT with the left qubit (q) as control."""
    g = np.eye(4, dtype=np.complex128)
    g[2:, 2:] = [[0, 1], [1, 0]]
    return g


def gate_cz() -> np.ndarray:
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def gate_swap() -> np.ndarray:
    g = np.zeros((4, 4), dtype=np.complex128)
    g[0, 0] = g[3, 3] = 1
    g[1, 2] = g[2, 1] = 1
    return g


def gate_rzz(t: float) -> np.ndarray:
    a, b = np.exp(-0.5j * t), np.exp(0.5j * t)
    return np.diag([a, b, b, a]).astype(np.complex128)


def gate_cp(phi: float) -> np.ndarray:
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def haar_su4(rng: np.random.Generator) -> np.ndarray:
    u = haar_unitary(4, rng)
    return u / np.linalg.det(u) ** 0.25


# --------------------------------------------------------------------------
# circuits


def _brick_pairs(n: int, t: int) -> np.ndarray:
    return np.arange(t % 2, n - 1, 2, dtype=np.int32)


def brickwork_su4(n: int, depth: int, seed: int) -> Circuit:
    """Haar SU(4) brickwork: layer t acts on pairs (q, q+1) with q = t mod 2, t mod 2 + 2, ..."""
    rng = np.random.default_rng(seed)
    layers = []
    for t in range(depth):
        pairs = _brick_pairs(n, t)
        g4 = np.stack([haar_su4(rng) for _ in pairs]) if len(pairs) else np.zeros((0, 4, 4))
        layers.append(Layer(pairs, g4))
    return Circuit(n, layers, {"kind": "brickwork_su4", "seed": seed, "depth": depth})


def brickwork_u2_su4(n: int, depth: int, seed: int) -> Circuit:
    """Brickwork whose every layer first applies Haar U(2) on every qubit, then Haar SU(4) pairs."""
    rng = np.random.default_rng(seed)
    layers = []
    for t in range(depth):
        u1 = np.stack([haar_unitary(2, rng) for _ in range(n)])
        pairs = _brick_pairs(n, t)
        g4 = np.stack([haar_su4(rng) for _ in pairs]) if len(pairs) else np.zeros((0, 4, 4))
        layers.append(Layer(pairs, g4, u1))
    return Circuit(n, layers, {"kind": "brickwork_u2_su4", "seed": seed, "depth": depth})


def gateset_circuit(n: int, depth: int, seed: int) -> Circuit:
    """Gate set {H, CX, RZZ(t), RX(t)}, t ~ U[0, 2pi), drawn uniformly per site.

    At layer t the pairs are at offset t mod 2.  For each pair one gate is drawn;
    a two-qubit draw (CX with the left qubit as control, or RZZ) acts on the pair,
    a one-qubit draw acts on the left qubit and an independent draw from {H, RX}
    acts on the right qubit.  A qubit outside every pair gets a draw from {H, RX}.
    """
    rng = np.random.default_rng(seed)

    def one_q():
        if rng.integers(2) == 0:
            return gate_h()
        return gate_rx(rng.uniform(0.0, 2 * np.pi))

    layers = []
    for t in range(depth):
        u1 = np.stack([np.eye(2, dtype=np.complex128)] * n)
        pairs, g4 = [], []
        covered = np.zeros(n, dtype=bool)
        for q in _brick_pairs(n, t):
            covered[q] = covered[q + 1] = True
            k = rng.integers(4)
            if k == 0:
                u1[q] = gate_h()
                u1[q + 1] = one_q()
            elif k == 1:
                pairs.append(q)
                g4.append(gate_cx())
            elif k == 2:
                pairs.append(q)
                g4.append(gate_rzz(rng.uniform(0.0, 2 * np.pi)))
            else:
                u1[q] = gate_rx(rng.uniform(0.0, 2 * np.pi))
                u1[q + 1] = one_q()
        for q in np.nonzero(~covered)[0]:
            u1[q] = one_q()
        g4a = np.stack(g4) if g4 else np.zeros((0, 4, 4), dtype=np.complex128)
        layers.append(Layer(np.array(pairs, dtype=np.int32), g4a, u1))
    return Circuit(n, layers, {"kind": "gateset", "seed": seed, "depth": depth})


def hea_circuit(n: int, n_layers: int, seed: int, sigma: float = 0.3):
    """Hardware-efficient ansatz: per layer RY(t), RZ(t) on every qubit, then a CZ ladder.

    The CZ ladder CZ(0,1), CZ(1,2), ... commutes, so it runs as an even and an odd
    sub-layer.  Returns (circuit, angles[n_layers, n, 2]).
    """
    rng = np.random.default_rng(seed)
    angles = rng.normal(0.0, sigma, size=(n_layers, n, 2))
    layers = []
    for l in range(n_layers):
        u1 = np.stack([gate_rz(angles[l, q, 1]) @ gate_ry(angles[l, q, 0]) for q in range(n)])
        for par in (0, 1):
            pairs = np.arange(par, n - 1, 2, dtype=np.int32)
            g4 = np.stack([gate_cz()] * len(pairs)) if len(pairs) else np.zeros((0, 4, 4))
            layers.append(Layer(pairs, g4, u1 if par == 0 else None))
    return Circuit(n, layers, {"kind": "hea", "seed": seed}), angles


def ghz_circuit(n: int) -> Circuit:
    """H on qubit 0, then CX(q, q+1) for q = 0 .. n-2, one gate per layer."""
    layers = []
    for q in range(n - 1):
        u1 = None
        if q == 0:
            u1 = np.stack([np.eye(2, dtype=np.complex128)] * n)
            u1[0] = gate_h()
        layers.append(Layer(np.array([q], dtype=np.int32), gate_cx()[None], u1))
    return Circuit(n, layers, {"kind": "ghz"})


def qft_nn_circuit(n: int, x_bits) -> Circuit:
    """Textbook QFT (no final bit reversal) on the basis state |x>, nearest-neighbour only.

    Input preparation puts X on the qubits with x_j = 1.  Logical qubit j gets H,
    then CP(2pi / 2^(k-j+1)) with every k > j.  A CP between qubits that are not
    adjacent is realised by moving k next to j with SWAP gates; at the end the
    qubits are bubble-sorted back into logical order, again with SWAPs.  Every gate
    is its own layer.
    """
    n = int(n)
    pos = list(range(n))        # logical -> physical
    at = list(range(n))         # physical -> logical
    layers: List[Layer] = []
    ident = np.stack([np.eye(2, dtype=np.complex128)] * n)

    def add_1q(phys, u):
        u1 = ident.copy()
        u1[phys] = u
        layers.append(Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4)), u1))

    def add_2q(p, g):
        layers.append(Layer(np.array([p], np.int32), g[None]))

    def swap_phys(p):
        add_2q(p, gate_swap())
        a, b = at[p], at[p + 1]
        at[p], at[p + 1] = b, a
        pos[a], pos[b] = p + 1, p

    u_prep = ident.copy()
    for j, b in enumerate(x_bits):
        if b:
            u_prep[j] = gate_x()
    layers.append(Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4)), u_prep))

    for j in range(n):
        add_1q(pos[j], gate_h())
        for k in range(j + 1, n):
            while abs(pos[k] - pos[j]) > 1:
                if pos[k] > pos[j]:
                    swap_phys(pos[k] - 1)
                else:
                    swap_phys(pos[k])
            p = min(pos[j], pos[k])
            add_2q(p, gate_cp(2 * np.pi / 2 ** (k - j + 1)))   # CP is symmetric
    changed = True
    while changed:
        changed = False
        for p in range(n - 1):
            if at[p] > at[p + 1]:
                swap_phys(p)
                changed = True
    return Circuit(n, layers, {"kind": "qft_nn", "x": list(map(int, x_bits))})


def batch_circuits(n_circ: int, base_seed: int = 1000):
    """Independent Haar SU(4) brickwork circuits of uneven width, depth and bond cap.

    Circuit i uses seed base_seed + i: width ~ U{16..128}, depth ~ U{8..32},
    chi_max ~ U{16, 32, 64, 128, 256}.  Returns a list of (circuit, chi_max).
    """
    out = []
    for i in range(n_circ):
        rng = np.random.default_rng(base_seed + i)
        n = int(rng.integers(16, 129))
        depth = int(rng.integers(8, 33))
        chi = int(rng.choice([16, 32, 64, 128, 256]))
        c = brickwork_su4(n, depth, base_seed + i)
        c.meta["chi_max"] = chi
        out.append((c, chi))
    return out


def nonlocal_ops(n: int, n_ops: int, seed: int, p1: float = 0.25, max_dist: Optional[int] = None):
    """A gate list on arbitrary qubits: with probability p1 a Haar U(2) on a uniform
    qubit, else a Haar U(4) on two distinct qubits at distance <= max_dist (default
    n - 1), in random order (either may be the first listed).  Items are
    (qa, qb, matrix) with qb None for one-qubit gates; a two-qubit matrix has basis
    index 2*b_qa + b_qb."""
    rng = np.random.default_rng(seed)
    dmax = n - 1 if max_dist is None else max(1, min(int(max_dist), n - 1))
    ops = []
    for _ in range(n_ops):
        if rng.random() < p1:
            ops.append((int(rng.integers(n)), None, haar_unitary(2, rng)))
            continue
        d = int(rng.integers(1, dmax + 1))
        lo = int(rng.integers(0, n - d))
        a, b = (lo, lo + d) if rng.random() < 0.5 else (lo + d, lo)
        ops.append((a, b, haar_unitary(4, rng)))
    return ops


def random_sites(chi_l: int, chi_m: int, chi_r: int, seed: int):
    """Two adjacent complex Gaussian site tensors (chi_l,2,chi_m), (chi_m,2,chi_r)."""
    rng = np.random.default_rng(seed)

    def cg(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)

    a = cg(chi_l, 2, chi_m) / np.sqrt(2 * chi_m)
    b = cg(chi_m, 2, chi_r) / np.sqrt(2 * chi_r)
    return a, b


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(count, n), dtype=np.uint8)


# --------------------------------------------------------------------------
# the named workloads


def config_c1(seed: int = 1):
    """10 qubits, depth 8, U(2) on every qubit then SU(4) pairs, chi_max 32 (exact), c128."""
    return brickwork_u2_su4(10, 8, seed), dict(chi_max=32, cutoff=0.0)


def config_c2(seed: int = 1, n: int = 64, depth: int = 20):
    """64 qubits, depth 20 Haar SU(4) brickwork, chi_max 128, cutoff 1e-10."""
    return brickwork_su4(n, depth, seed), dict(chi_max=128, cutoff=1e-10)


def config_c3(seed: int = 1, n: int = 100, depth: int = 24):
    """100 qubits, depth 24, gate set {H, CX, RZZ, RX}, chi_max 256."""
    return gateset_circuit(n, depth, seed), dict(chi_max=256, cutoff=0.0)
