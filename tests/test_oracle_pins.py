"""Pins of the FP64 oracle against things other than itself (CPU only).

* brute force: the dense state-vector simulator (full contraction, Eq. 1) at
  <= 10 qubits, where an MPS with an untruncated bond is exact;
* closed forms: GHZ (Sec. V.A), the QFT of a basis state (uniform magnitudes
  2^(-n/2) with known phases), product states;
* invariants: unit norm, left isometries of freshly written left sites,
  canonical forms, sum of s^2 = |theta|_F^2, 1q-only layers keep the bonds;
* designed spectra for the truncation rule, and the dense Schmidt truncation at
  a cut for the truncated update in mixed-canonical gauge.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense
from oracle import mps as om

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_bits(n):
    return [[(x >> (n - 1 - i)) & 1 for i in range(n)] for x in range(2 ** n)]


# ----------------------------------------------------------------- brute force


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_c1_exact_mps_equals_dense(seed):
    """10 qubits, depth 8, chi_max 32 = 2^(n/2): no truncation, every amplitude exact."""
    circ, p = W.config_c1(seed)
    m, recs = om.run_circuit(circ, p["chi_max"], p["cutoff"])
    psi = dense.run_circuit(circ)
    got = om.to_dense(m)
    assert np.max(np.abs(got - psi)) < 1e-12
    amps = om.amplitudes(m, _all_bits(10)[::37])
    assert np.max(np.abs(amps - psi[::37])) < 1e-12
    assert max(r.eps for rr in recs for r in rr) < 1e-24
    assert max(m.bond_dims()) <= 32


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_every_gate_position_small(n):
    rng = np.random.default_rng(100 + n)
    m = om.zero_state(n)
    psi = dense.zero_state(n)
    for q in range(n):
        u = W.haar_unitary(2, rng)
        om.apply_1q(m, q, u)
        psi = dense.apply_1q(psi, n, q, u)
    for rep in range(3):
        for q in range(n - 1):
            g = W.haar_unitary(4, rng)
            om.apply_2q(m, q, g, chi_max=2 ** n)
            psi = dense.apply_2q(psi, n, q, g)
    assert np.max(np.abs(om.to_dense(m) - psi)) < 1e-12


def test_gate_index_convention_cx():
    """CX with the left qubit as control flips the right qubit only when the left is 1."""
    for x0 in (0, 1):
        for x1 in (0, 1):
            m = om.zero_state(2)
            if x0:
                om.apply_1q(m, 0, W.gate_x())
            if x1:
                om.apply_1q(m, 1, W.gate_x())
            om.apply_2q(m, 0, W.gate_cx(), chi_max=4)
            want = [x0, x1 ^ x0]
            assert abs(om.amplitude(m, want) - 1) < 1e-14


# ----------------------------------------------------------------- closed forms


def test_ghz_golden():
    gold = json.load(open(os.path.join(GOLDEN, "ghz.json")))
    a = gold["nonzero_amplitude"]
    for n in gold["widths"]:
        m, _ = om.run_circuit(W.ghz_circuit(n), chi_max=64)
        assert max(m.bond_dims()) == gold["max_bond_dimension"]
        assert abs(om.amplitude(m, [0] * n) - a) < 1e-14
        assert abs(om.amplitude(m, [1] * n) - a) < 1e-14
        rng = np.random.default_rng(n)
        for bits in rng.integers(0, 2, size=(20, n)):
            if 0 < bits.sum() < n:
                assert abs(om.amplitude(m, bits)) < 1e-14


@pytest.mark.parametrize("n,seed", [(4, 1), (6, 2), (7, 3)])
def test_qft_basis_state_closed_form(n, seed):
    """QFT (no final reversal) of |x>: qubit j ends in (|0> + e^{2 pi i 0.x_j...x_{n-1}}|1>)/sqrt 2."""
    x = np.random.default_rng(seed).integers(0, 2, size=n)
    m, _ = om.run_circuit(W.qft_nn_circuit(n, x), chi_max=2 ** n)
    assert max(m.bond_dims()) == 1            # a product state throughout
    for z in _all_bits(n):
        ph = sum(z[j] * sum(x[k] * 2.0 ** (-(k - j + 1)) for k in range(j, n)) for j in range(n))
        want = np.exp(2j * np.pi * ph) / 2 ** (n / 2)
        assert abs(om.amplitude(m, z) - want) < 1e-13


def test_product_state_z():
    n = 7
    bits = [1, 0, 0, 1, 1, 0, 1]
    m = om.zero_state(n)
    for q, b in enumerate(bits):
        if b:
            om.apply_1q(m, q, W.gate_x())
    for q, b in enumerate(bits):
        p = "I" * q + "Z" + "I" * (n - q - 1)
        assert abs(om.expect_pauli(m, p) - (1 - 2 * b)) < 1e-15


# ----------------------------------------------------------------- invariants


def test_unit_norm_and_left_isometry():
    circ, p = W.config_c1(3)
    m = om.zero_state(circ.n_qubits)
    for layer in circ.layers:
        recs = om.apply_layer(m, layer, p["chi_max"])
        for r in recs:
            a = m.sites[r.q]
            mat = a.reshape(-1, a.shape[2])
            assert np.max(np.abs(mat.conj().T @ mat - np.eye(a.shape[2]))) < 1e-12
    assert abs(om.norm2(m) - 1.0) < 1e-12
    assert abs(np.vdot(om.to_dense(m), om.to_dense(m)) - om.norm2(m)) < 1e-12


def test_sum_s2_is_theta_frobenius():
    """Sigma s^2 = |theta|_F^2, with theta taken from the dense state in mixed gauge.

    After left-canonicalising sites < q and right-canonicalising sites > q+1 the
    Frobenius norm of theta is the norm of the whole state (taken from the dense
    simulator, which shares nothing with the MPS update).
    """
    circ, p = W.config_c1(2)
    m, _ = om.run_circuit(circ, p["chi_max"])
    psi = dense.run_circuit(circ)
    g = W.haar_su4(np.random.default_rng(9))
    q = 4
    lc = om.left_canonicalize(m)
    rc = om.right_canonicalize(lc)   # sites 1..n-1 right-isometric, site 0 holds the norm
    mixed = om.left_canonicalize(om.MPS(rc.sites[: q + 1]))  # sites 0..q-1 left iso
    sites = mixed.sites[:q] + [mixed.sites[q]] + rc.sites[q + 1:]
    mm = om.MPS(sites)
    rec = om.apply_2q(mm, q, g, chi_max=1024)
    psi2 = dense.apply_2q(psi, circ.n_qubits, q, g)
    assert abs(np.sum(rec.s_all ** 2) - np.vdot(psi2, psi2).real) < 1e-12


def test_one_qubit_layer_keeps_bonds():
    circ, p = W.config_c1(4)
    m, _ = om.run_circuit(circ, p["chi_max"])
    before = m.bond_dims()
    rng = np.random.default_rng(0)
    u1 = np.stack([W.haar_unitary(2, rng) for _ in range(circ.n_qubits)])
    om.apply_layer(m, W.Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4)), u1), p["chi_max"])
    assert m.bond_dims() == before


def test_identity_and_swap_twice():
    circ, p = W.config_c1(5)
    m, _ = om.run_circuit(circ, p["chi_max"])
    ref = m.copy()
    for q in range(0, 9, 2):
        om.apply_2q(m, q, np.eye(4, dtype=complex), chi_max=32)
    assert abs(om.fidelity(m, ref) - 1) < 1e-12
    for q in (1, 5):
        om.apply_2q(m, q, W.gate_swap(), chi_max=32)
        om.apply_2q(m, q, W.gate_swap(), chi_max=32)
    assert np.max(np.abs(om.to_dense(m) - om.to_dense(ref))) < 1e-12


def test_canonical_forms():
    circ, p = W.config_c1(1)
    m, _ = om.run_circuit(circ, p["chi_max"])
    psi = om.to_dense(m)
    lc = om.left_canonicalize(m)
    rc = om.right_canonicalize(m)
    for a in lc.sites[:-1]:
        mat = a.reshape(-1, a.shape[2])
        assert np.max(np.abs(mat.conj().T @ mat - np.eye(mat.shape[1]))) < 1e-12
    for a in rc.sites[1:]:
        mat = a.reshape(a.shape[0], -1)
        assert np.max(np.abs(mat @ mat.conj().T - np.eye(mat.shape[0]))) < 1e-12
    assert np.max(np.abs(om.to_dense(lc) - psi)) < 1e-12
    assert np.max(np.abs(om.to_dense(rc) - psi)) < 1e-12


def test_expectations_and_overlap_vs_dense():
    circ, p = W.config_c1(2)
    m, _ = om.run_circuit(circ, p["chi_max"])
    psi = dense.run_circuit(circ)
    n = circ.n_qubits
    rng = np.random.default_rng(4)
    for _ in range(12):
        ps = "".join(rng.choice(list("IXYZ"), size=n))
        assert abs(om.expect_pauli(m, ps) - dense.expect_pauli(psi, n, ps)) < 1e-12
    circ2, _ = W.config_c1(3)
    m2, _ = om.run_circuit(circ2, 32)
    psi2 = dense.run_circuit(circ2)
    assert abs(om.overlap(m, m2) - np.vdot(psi, psi2)) < 1e-12


def test_perfect_sampling_distribution():
    circ = W.brickwork_u2_su4(4, 4, seed=7)
    m, _ = om.run_circuit(circ, 16)
    probs = np.abs(dense.run_circuit(circ)) ** 2
    shots = om.perfect_sample(m, 20000, np.random.default_rng(1))
    idx = shots.astype(np.int64) @ (1 << np.arange(3, -1, -1))
    freq = np.bincount(idx, minlength=16) / len(shots)
    assert 0.5 * np.sum(np.abs(freq - probs)) < 0.02
    assert np.all(probs[np.unique(idx)] > 0)


# ----------------------------------------------------------------- truncation


def _designed_sites(s, seed):
    """Two sites whose theta (for the identity gate) has singular values s exactly."""
    rng = np.random.default_rng(seed)
    r = len(s)
    chi = r // 2
    u = W.haar_unitary(r, rng)
    v = W.haar_unitary(r, rng)
    theta = (u * np.asarray(s)[None, :]) @ v.conj().T            # (2chi) x (2chi)
    a = u.reshape(chi, 2, r)                                      # chi_L = chi, bond r
    b = ((np.asarray(s)[:, None]) * v.conj().T).reshape(r, 2, chi)
    return a, b, theta


@pytest.mark.parametrize("chi_max,cutoff,want_k", [
    (16, 0.0, 12),     # 4 exact zeros dropped
    (8, 0.0, 8),       # bond cap binds
    (16, 1e-3, 8),     # cutoff binds: tail from 8 on is 6.8e-4 of the total, from 7 on 1.9e-3
    (16, 1e-1, 4),
    (1, 0.0, 1),
])
def test_truncation_rank_designed(chi_max, cutoff, want_k):
    s = np.array([1.0, 0.8, 0.5, 0.4, 0.2, 0.1, 0.07, 0.05, 0.03, 0.02, 0.01, 0.005,
                  0, 0, 0, 0])
    tot = np.sum(s * s)
    k, eps = om.truncation_rank(s, 16, 16, chi_max, cutoff)
    assert k == want_k
    assert eps == pytest.approx(np.sum(s[k:] ** 2) / tot, rel=1e-14, abs=1e-300)


def test_truncated_update_is_eckart_young():
    s = np.sort(np.random.default_rng(3).uniform(0.01, 1, 16))[::-1]
    a, b, theta = _designed_sites(s, 11)
    m = om.MPS([a, b])
    rec = om.apply_2q(m, 0, np.eye(4, dtype=complex), chi_max=5, renormalize=False)
    assert rec.k == 5
    assert np.allclose(rec.s_all, s, atol=1e-14, rtol=0)
    approx = np.einsum("lxb,byr->lxyr", m.sites[0], m.sites[1]).reshape(theta.shape)
    err = np.linalg.norm(theta - approx) ** 2
    assert err == pytest.approx(np.sum(s[5:] ** 2), rel=1e-10)
    assert rec.eps == pytest.approx(np.sum(s[5:] ** 2) / np.sum(s ** 2), rel=1e-12)


@pytest.mark.parametrize("q,k", [(2, 3), (3, 5), (1, 2)])
def test_truncated_update_matches_dense_schmidt_cut(q, k):
    """In mixed-canonical gauge the truncated pair update equals the dense state's
    best rank-k Schmidt approximation across the cut (q | q+1), renormalised."""
    n = 7
    circ = W.brickwork_u2_su4(n, 6, seed=21)
    m, _ = om.run_circuit(circ, 2 ** n)
    psi = dense.run_circuit(circ)
    rc = om.right_canonicalize(m)
    head = om.left_canonicalize(om.MPS(rc.sites[: q + 1]))
    mm = om.MPS(head.sites + rc.sites[q + 1:])
    g = W.haar_su4(np.random.default_rng(q))
    om.apply_2q(mm, q, g, chi_max=k, renormalize=True)
    psi2 = dense.apply_2q(psi, n, q, g).reshape(2 ** (q + 1), -1)
    u, s, vh = np.linalg.svd(psi2, full_matrices=False)
    sk = s[:k] * np.sqrt(np.sum(s ** 2) / np.sum(s[:k] ** 2))
    want = ((u[:, :k] * sk[None, :]) @ vh[:k]).reshape(-1)
    assert np.max(np.abs(om.to_dense(mm) - want)) < 1e-12
    assert mm.bond_dims()[q + 1] == k


def test_svd_step_properties():
    """The library SVD returns a true decomposition: orthonormal factors, descending s."""
    a, b = W.random_sites(6, 9, 5, seed=2)
    g = W.haar_su4(np.random.default_rng(2))
    theta = om.contract_gate(om.merge_sites(a, b), g).reshape(12, 10)
    u, s, vh = np.linalg.svd(theta, full_matrices=False)
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert np.max(np.abs(u.conj().T @ u - np.eye(10))) < 1e-13
    assert np.max(np.abs(vh @ vh.conj().T - np.eye(10))) < 1e-13
    assert np.max(np.abs((u * s) @ vh - theta)) < 1e-13


# ----------------------------------------------------------------- the complex64 precision floor


def test_single_precision_floor_variant():
    """apply_2q_single_precision: the paper's update with complex64 storage and
    contraction around an exact SVD.  Pins: exact on data whose products are exact in
    single precision (CX on basis states), within single-precision rounding of the
    dense state vector on the exact 10-qubit circuit (and measurably not FP64, so
    the rounding is really applied), and every stored site representable in complex64."""
    # CX (control = left) on |10>: theta entries are 0 and 1, so nothing rounds
    for single in (False, True):
        m = om.zero_state(4)
        om.apply_1q(m, 1, W.gate_x())
        upd = om.apply_2q_single_precision if single else om.apply_2q
        upd(m, 1, W.gate_cx(), 4)
        bits = np.array([[0, 1, 1, 0], [0, 1, 0, 0]], dtype=np.uint8)
        amps = om.amplitudes(m, bits)
        assert abs(amps[0] - 1) < 1e-15 and abs(amps[1]) < 1e-15
    # the exact C1 circuit, layer by layer
    circ, p = W.config_c1(2)
    m64, _ = om.run_circuit(circ, p["chi_max"])
    m32, _ = om.run_circuit(circ, p["chi_max"], single=True)
    psi = dense.run_circuit(circ)
    d32 = om.to_dense(m32)
    err = np.linalg.norm(d32 - psi) / np.linalg.norm(psi)
    assert 1e-9 < err < 1e-5
    assert np.linalg.norm(om.to_dense(m64) - psi) < 1e-12
    for s in m32.sites:
        assert np.array_equal(s, s.astype(np.complex64).astype(np.complex128))
