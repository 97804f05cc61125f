"""FP64 Matrix Product State simulator -- the oracle of the two-qubit gate path.

Test infrastructure only (see the package docstring).  Every site tensor is
complex128 with shape (chi_q, 2, chi_{q+1}) (Eq. 2: one physical leg, two bond
legs; the terminal sites have a bond of dimension one).

The two-qubit update follows Sec. III.A "Two Qubit Gate" and Sec. IV.A
(``simulation_kernel``) step by step:

1. merge the two sites over their shared bond (Fig. 2, "merge two tensors"):
   ``M[l, p0, p1, r] = sum_b A_q[l, p0, b] A_{q+1}[b, p1, r]``;
2. contract the gate, cast as a 2x2x2x2 tensor (Eq. 1 and Sec. III.A "Non-local"
   paragraph, first sentence): ``theta[l, a, b, r] = sum_{c,d} G[a, b, c, d] M[l, c, d, r]``;
3. SVD of theta viewed as the (2 chi_L) x (2 chi_R) matrix with rows (l, a) and
   columns (b, r), with the bond truncated (Sec. II.A best low-rank approximation;
   Sec. IV.A "the bond dimension can be truncated");
4. the left singular vectors become the left ("control") site and the right
   singular vectors with the singular values contracted in become the right
   ("target") site (Sec. III.A "Two Qubit Gate").

Readings where the paper is silent:

* truncation rank: singular values below ``eps * max(m, n) * s_max`` are treated
  as exact zeros; then k = min(chi_max, #nonzero, smallest k whose discarded
  weight sum_{j>=k} s_j^2 is <= cutoff * sum_j s_j^2), and k >= 1;
* the discarded weight reported per gate is that relative sum;
* when ``renormalize`` is set, the kept singular values are scaled so that their
  squares sum to sum_j s_j^2 of the untruncated theta;
* the S factor always goes to the right site of the pair, whatever the gate.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

EPS64 = float(np.finfo(np.float64).eps)

PAULI = {
    "I": np.array([[1, 0], [0, 1]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


@dataclass
class GateRecord:
    """What one two-qubit update produced (for comparisons with the CUDA path)."""

    q: int
    s_all: np.ndarray      # every singular value of theta, descending
    k: int                 # kept bond dimension
    eps: float             # relative discarded weight
    s_kept: np.ndarray     # kept singular values after optional renormalisation


class MPS:
    def __init__(self, sites: List[np.ndarray]):
        self.sites = [np.asarray(s, dtype=np.complex128) for s in sites]
        # the singular values written by the last SVD on each bond (bond b sits
        # between sites b-1 and b); None for bonds no SVD has touched
        self.spectrum: List[Optional[np.ndarray]] = [None] * (len(self.sites) + 1)

    @property
    def n(self) -> int:
        return len(self.sites)

    def bond_dims(self) -> List[int]:
        return [1] + [s.shape[2] for s in self.sites]

    def copy(self) -> "MPS":
        m = MPS([s.copy() for s in self.sites])
        m.spectrum = [None if x is None else x.copy() for x in self.spectrum]
        return m


# --------------------------------------------------------------------------
# state and gates


def zero_state(n: int) -> MPS:
    """|0...0> with every bond of dimension one (Sec. IV.A "Implementations")."""
    sites = []
    for _ in range(n):
        a = np.zeros((1, 2, 1), dtype=np.complex128)
        a[0, 0, 0] = 1.0
        sites.append(a)
    return MPS(sites)


def apply_1q(mps: MPS, q: int, u: np.ndarray) -> None:
    """A'[l, p', r] = sum_p U[p', p] A[l, p, r]  (Eq. 3); no other site changes."""
    mps.sites[q] = np.einsum("ab,lbr->lar", u, mps.sites[q])


def merge_sites(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """M[l, p0, p1, r] = sum_b A[l, p0, b] B[b, p1, r]  (Fig. 2)."""
    return np.einsum("lxb,byr->lxyr", a, b)


def contract_gate(m: np.ndarray, g: np.ndarray) -> np.ndarray:
    """theta[l, a, b, r] = sum_{c,d} G[a, b, c, d] M[l, c, d, r], G = g as 2x2x2x2 (Eq. 1)."""
    G = g.reshape(2, 2, 2, 2)
    return np.einsum("abcd,lcdr->labr", G, m)


def truncation_rank(s: np.ndarray, m: int, n: int, chi_max: int, cutoff: float,
                    eps: float = EPS64):
    """Kept rank k and relative discarded weight for descending singular values s.

    Returns (k, discarded_weight).  ``eps`` is the unit of the arithmetic that
    produced s (float64 here); values below eps * max(m, n) * s_max are zeros.
    """
    s = np.asarray(s, dtype=np.float64)
    total = float(np.sum(s * s))
    if total == 0.0:
        return 1, 0.0
    s_max = float(s[0])
    nonzero = int(np.count_nonzero(s > eps * max(m, n) * s_max))
    k = max(1, min(int(chi_max), nonzero))
    if cutoff > 0.0:
        # smallest kk whose tail weight sum_{j >= kk} s_j^2 is within the cutoff
        tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
        kk = int(np.argmax(tail <= cutoff * total))
        k = max(1, min(k, kk))
    disc = float(np.sum(s[k:] * s[k:])) / total
    return k, disc


def apply_2q(mps: MPS, q: int, g: np.ndarray, chi_max: int, cutoff: float = 0.0,
             renormalize: bool = True) -> GateRecord:
    """Local two-qubit gate on sites (q, q+1): merge, gate, truncated SVD, absorb."""
    a, b = mps.sites[q], mps.sites[q + 1]
    chi_l, chi_r = a.shape[0], b.shape[2]
    theta = contract_gate(merge_sites(a, b), g)
    mat = theta.reshape(2 * chi_l, 2 * chi_r)
    u, s, vh = np.linalg.svd(mat, full_matrices=False)        # LAPACK, descending s
    k, disc = truncation_rank(s, mat.shape[0], mat.shape[1], chi_max, cutoff)
    s_kept = s[:k].copy()
    if renormalize:
        kept = float(np.sum(s_kept ** 2))
        if kept > 0.0:
            s_kept *= np.sqrt(float(np.sum(s * s)) / kept)
    mps.sites[q] = u[:, :k].reshape(chi_l, 2, k)
    mps.sites[q + 1] = (s_kept[:, None] * vh[:k, :]).reshape(k, 2, chi_r)
    mps.spectrum[q + 1] = s_kept.copy()
    return GateRecord(q, s, k, disc, s_kept)


def apply_2q_canonical(mps: MPS, q: int, g: np.ndarray, chi_max: int, cutoff: float = 0.0,
                       renormalize: bool = True) -> GateRecord:
    """Local two-qubit gate with the state kept in right-canonical form and the
    singular values of every bond stored beside it (Hastings, "Light-cone matrix
    product", J. Math. Phys. 50, 095207 (2009)).

    With Lam the singular values of bond q (those of the last SVD there; ones for a
    bond no SVD has touched) and theta the gate applied to the merged sites as in
    apply_2q:
      * the SVD is taken of diag(Lam) theta (rows (l, a) scaled by Lam[l]), whose
        singular values are the Schmidt coefficients of the cut q+1, so truncation
        acts on them;
      * the right site becomes V^H (k rows), the left site theta V -- without
        dividing by Lam -- times the renormalisation factor;
      * bond q+1 stores the kept (renormalised) singular values.
    """
    a, b = mps.sites[q], mps.sites[q + 1]
    chi_l, chi_r = a.shape[0], b.shape[2]
    lam = mps.spectrum[q] if mps.spectrum[q] is not None else np.ones(chi_l)
    assert lam.shape[0] == chi_l
    theta = contract_gate(merge_sites(a, b), g)
    mat0 = theta.reshape(2 * chi_l, 2 * chi_r)
    mat = (lam[:, None, None, None] * theta).reshape(2 * chi_l, 2 * chi_r)
    u, s, vh = np.linalg.svd(mat, full_matrices=False)
    k, disc = truncation_rank(s, mat.shape[0], mat.shape[1], chi_max, cutoff)
    s_kept = s[:k].copy()
    scale = 1.0
    if renormalize:
        kept = float(np.sum(s_kept ** 2))
        if kept > 0.0:
            scale = np.sqrt(float(np.sum(s * s)) / kept)
    s_kept *= scale
    vk = vh[:k, :]
    mps.sites[q] = (scale * (mat0 @ vk.conj().T)).reshape(chi_l, 2, k)
    mps.sites[q + 1] = vk.reshape(k, 2, chi_r)
    mps.spectrum[q + 1] = s_kept.copy()
    return GateRecord(q, s, k, disc, s_kept)


def apply_2q_single_precision(mps: MPS, q: int, g: np.ndarray, chi_max: int, cutoff: float = 0.0,
                              renormalize: bool = True) -> GateRecord:
    """apply_2q with the storage and contraction precision of a complex64 run and an
    exact SVD: the precision floor of any complex64 path.

    Both sites are read as complex64, the merge (Fig. 2) is a complex64 matrix product
    and the gate (Eq. 1) a complex64 contraction, both accumulating in single
    precision; theta is then decomposed in FP64 (LAPACK), truncated with the
    single-precision zero threshold (eps = eps_32), and the new sites are rounded to
    complex64.  Comparing a complex64 path with apply_2q measures its whole error;
    comparing this function with apply_2q measures the part that no SVD, however
    accurate, can remove."""
    a = mps.sites[q].astype(np.complex64)
    b = mps.sites[q + 1].astype(np.complex64)
    chi_l, chi_m, chi_r = a.shape[0], a.shape[2], b.shape[2]
    merged = (a.reshape(2 * chi_l, chi_m) @ b.reshape(chi_m, 2 * chi_r)).reshape(chi_l, 2, 2, chi_r)
    G = g.astype(np.complex64).reshape(2, 2, 2, 2)
    theta = np.einsum("abcd,lcdr->labr", G, merged)
    mat = theta.reshape(2 * chi_l, 2 * chi_r).astype(np.complex128)
    u, s, vh = np.linalg.svd(mat, full_matrices=False)
    k, disc = truncation_rank(s, mat.shape[0], mat.shape[1], chi_max, cutoff,
                              eps=float(np.finfo(np.float32).eps))
    s_kept = s[:k].copy()
    if renormalize:
        kept = float(np.sum(s_kept ** 2))
        if kept > 0.0:
            s_kept *= np.sqrt(float(np.sum(s * s)) / kept)
    left = u[:, :k].reshape(chi_l, 2, k)
    right = (s_kept[:, None] * vh[:k, :]).reshape(k, 2, chi_r)
    mps.sites[q] = left.astype(np.complex64).astype(np.complex128)
    mps.sites[q + 1] = right.astype(np.complex64).astype(np.complex128)
    mps.spectrum[q + 1] = s_kept.copy()
    return GateRecord(q, s, k, disc, s_kept)


def apply_layer(mps: MPS, layer, chi_max: int, cutoff: float = 0.0,
                renormalize: bool = True, canonical: bool = False, single: bool = False) -> List[GateRecord]:
    """One layer: its one-qubit gates on every qubit, then its disjoint two-qubit gates
    (apply_2q, apply_2q_canonical when ``canonical``, or apply_2q_single_precision when
    ``single``)."""
    if layer.u1 is not None:
        for q in range(mps.n):
            apply_1q(mps, q, layer.u1[q])
            if single:   # complex64 storage
                mps.sites[q] = mps.sites[q].astype(np.complex64).astype(np.complex128)
    upd = apply_2q_canonical if canonical else apply_2q
    if single:
        upd = apply_2q_single_precision
    recs = []
    for q, g in zip(layer.pairs, layer.g4):
        recs.append(upd(mps, int(q), g, chi_max, cutoff, renormalize))
    return recs


# SWAP on an adjacent pair in the basis 2 b_q + b_{q+1}
SWAP = np.array([[1, 0, 0, 0],
                 [0, 0, 1, 0],
                 [0, 1, 0, 0],
                 [0, 0, 0, 1]], dtype=np.complex128)


def reversed_pair(g: np.ndarray) -> np.ndarray:
    """The 4x4 of the same gate with its two qubits named in the other order:
    as a tensor G[a, b, c, d] (outputs a, b; inputs c, d) both pairs of legs swap."""
    return g.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)


def apply_2q_any(mps: MPS, qa: int, qb: int, g: np.ndarray, chi_max: int, cutoff: float = 0.0,
                 renormalize: bool = True, canonical: bool = False) -> List[GateRecord]:
    """Two-qubit gate on any two distinct qubits by the SWAP method (Sec. IV.B
    simulation_kernel: SWAP gates make the distant sites local, the gate is applied,
    and the SWAPs are reversed).  ``g`` has basis index 2*b_qa + b_qb.

    Reading of "move the distant sites": the qubit farther right, hi, moves left by
    SWAPs on (hi-1, hi), (hi-2, hi-1), ..., (lo+1, lo+2) until it sits at lo+1; the
    gate acts on (lo, lo+1); the same SWAPs then run in reverse order.  Every SWAP is
    an ordinary truncating two-qubit update.  Returns one record per update."""
    if qa == qb:
        raise ValueError("the two qubits must differ")
    lo, hi, gl = (qa, qb, g) if qa < qb else (qb, qa, reversed_pair(g))
    upd = apply_2q_canonical if canonical else apply_2q
    recs = []
    for j in range(hi - 1, lo, -1):
        recs.append(upd(mps, j, SWAP, chi_max, cutoff, renormalize))
    recs.append(upd(mps, lo, gl, chi_max, cutoff, renormalize))
    for j in range(lo + 1, hi):
        recs.append(upd(mps, j, SWAP, chi_max, cutoff, renormalize))
    return recs


def run_ops(n: int, ops, chi_max: int, cutoff: float = 0.0, renormalize: bool = True,
            mps: Optional[MPS] = None, canonical: bool = False):
    """Apply a gate list in program order from |0...0> (or from ``mps``).  ``ops`` holds
    (qa, qb, matrix) with qb None or negative for a one-qubit gate.  Returns
    (mps, records of every two-qubit update, SWAPs included)."""
    if mps is None:
        mps = zero_state(n)
    recs = []
    for qa, qb, g in ops:
        g = np.asarray(g, dtype=np.complex128)
        if qb is None or qb < 0:
            apply_1q(mps, int(qa), g)
        else:
            recs += apply_2q_any(mps, int(qa), int(qb), g, chi_max, cutoff, renormalize, canonical)
    return mps, recs


def run_circuit(circuit, chi_max: int, cutoff: float = 0.0, renormalize: bool = True,
                mps: Optional[MPS] = None, canonical: bool = False, single: bool = False):
    """Run every layer from |0...0> (or from ``mps``); returns (mps, records per layer)."""
    if mps is None:
        mps = zero_state(circuit.n_qubits)
    recs = [apply_layer(mps, layer, chi_max, cutoff, renormalize, canonical, single) for layer in circuit.layers]
    return mps, recs


# --------------------------------------------------------------------------
# read-out


def amplitude(mps: MPS, bits) -> complex:
    """<x|psi> = A_0[x_0] A_1[x_1] ... A_{n-1}[x_{n-1}]  (Eq. 2 with fixed physical legs)."""
    v = np.ones((1,), dtype=np.complex128)
    for a, x in zip(mps.sites, bits):
        v = v @ a[:, int(x), :]
    return complex(v[0])


def amplitudes(mps: MPS, bitstrings) -> np.ndarray:
    return np.array([amplitude(mps, b) for b in bitstrings], dtype=np.complex128)


def _transfer(sites_bra, sites_ket, ops=None) -> complex:
    """sum over all physical legs of conj(bra) (x) op (x) ket, left to right."""
    e = np.ones((1, 1), dtype=np.complex128)
    for i, (a, b) in enumerate(zip(sites_bra, sites_ket)):
        op = np.eye(2, dtype=np.complex128) if ops is None else ops[i]
        # e'[a', b'] = sum conj(A[x, p, a']) op[p, p'] e[x, y] B[y, p', b']
        t = np.einsum("xy,ypb->xpb", e, b)
        t = np.einsum("qp,xpb->xqb", op, t)
        e = np.einsum("xqa,xqb->ab", a.conj(), t)
    return complex(e[0, 0])


def overlap(bra: MPS, ket: MPS) -> complex:
    """<bra|ket> by a left-to-right transfer-matrix contraction."""
    return _transfer(bra.sites, ket.sites)


def norm2(mps: MPS) -> float:
    return float(overlap(mps, mps).real)


def fidelity(a: MPS, b: MPS) -> float:
    """|<a|b>|^2 / (<a|a><b|b>)."""
    ov = overlap(a, b)
    return float(abs(ov) ** 2 / (norm2(a) * norm2(b)))


def expect_pauli(mps: MPS, pstring: str) -> complex:
    """<psi| P_0 (x) ... (x) P_{n-1} |psi> for a string over {I, X, Y, Z}."""
    ops = [PAULI[c] for c in pstring]
    return _transfer(mps.sites, mps.sites, ops)


def to_dense(mps: MPS) -> np.ndarray:
    """Contract the whole chain into a 2^n vector (small n only)."""
    t = mps.sites[0]
    for a in mps.sites[1:]:
        t = np.tensordot(t, a, axes=([t.ndim - 1], [0]))
    return t.reshape(-1)


# --------------------------------------------------------------------------
# canonical forms and sampling (Sec. IV.A "Measurement operations", Sec. III.A "Sampling")


def left_canonicalize(mps: MPS) -> MPS:
    """QR sweep left to right: every site but the last becomes a left isometry."""
    out = mps.copy()
    for q in range(out.n - 1):
        a = out.sites[q]
        cl, _, cr = a.shape
        qm, r = np.linalg.qr(a.reshape(cl * 2, cr))
        out.sites[q] = qm.reshape(cl, 2, qm.shape[1])
        out.sites[q + 1] = np.einsum("ab,bpr->apr", r, out.sites[q + 1])
    return out


def right_canonicalize(mps: MPS) -> MPS:
    """QR sweep right to left on the conjugate transpose: sites 1..n-1 become right isometries."""
    out = mps.copy()
    for q in range(out.n - 1, 0, -1):
        a = out.sites[q]
        cl, _, cr = a.shape
        qm, r = np.linalg.qr(a.reshape(cl, 2 * cr).conj().T)     # a = r^H qm^H
        out.sites[q] = qm.conj().T.reshape(qm.shape[1], 2, cr)
        out.sites[q - 1] = np.einsum("lpb,bc->lpc", out.sites[q - 1], r.conj().T)
    return out


def perfect_sample_u(mps: MPS, u: np.ndarray) -> np.ndarray:
    """Perfect sampling (Sec. III.A "Sampling"; Sec. IV.A: canonicalise, then sample)
    with the random draws given: shot s takes bit b_q = 1 exactly when
    u[s, q] * (p0 + p1) >= p0, where p0, p1 are the weights of the two outcomes of
    qubit q given the bits already drawn.  After each draw the prefix is projected on
    its outcome and renormalised.  Plain version: no memoisation.  Returns uint8
    [n_shots, n]."""
    u = np.asarray(u, dtype=np.float64)
    rc = right_canonicalize(mps)
    nrm = np.sqrt(norm2(rc))
    out = np.zeros((u.shape[0], rc.n), dtype=np.uint8)
    for s in range(u.shape[0]):
        v = np.ones((1,), dtype=np.complex128) / nrm
        for q, a in enumerate(rc.sites):
            w0 = v @ a[:, 0, :]
            w1 = v @ a[:, 1, :]
            p0 = float(np.vdot(w0, w0).real)
            p1 = float(np.vdot(w1, w1).real)
            b = 1 if u[s, q] * (p0 + p1) >= p0 else 0
            w, p = (w1, p1) if b else (w0, p0)
            v = w / np.sqrt(p)
            out[s, q] = b
    return out


def perfect_sample(mps: MPS, n_shots: int, rng: np.random.Generator) -> np.ndarray:
    """perfect_sample_u with uniforms drawn from rng (row by row, qubit 0 first)."""
    return perfect_sample_u(mps, rng.random((n_shots, mps.n)))
