"""Pins of the oracle's canonical-form update (apply_2q_canonical, Hastings form).

* untruncated runs equal the dense contraction, every stored bond spectrum equals
  the Schmidt coefficients of the dense state at that cut (SVD of the reshaped
  vector), and every site right of the first is a right isometry;
* one truncation of an exact canonical state keeps the fraction of the state
  that Eckart-Young fixes for a Schmidt cut: F = sum_kept s^2 / sum s^2;
* SWAP chains in canonical form equal the dense contraction.
"""
import numpy as np
import pytest

import oracle.dense as D
import oracle.mps as M
import workloads as W


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_untruncated_equals_dense_with_schmidt_spectra(seed):
    circ, p = W.config_c1(seed)
    n = circ.n_qubits
    m, _ = M.run_circuit(circ, p["chi_max"], canonical=True)
    psi = D.run_circuit(circ)
    assert np.max(np.abs(M.to_dense(m) - psi)) < 1e-12
    for b in range(1, n):
        sv = np.linalg.svd(psi.reshape(2 ** b, -1), compute_uv=False)
        lam = m.spectrum[b]
        assert lam is not None
        assert np.max(np.abs(sv[: len(lam)] - lam)) < 1e-12 and np.all(sv[len(lam):] < 1e-12)
    for a in m.sites[1:]:
        assert np.max(np.abs(np.einsum("lpr,mpr->lm", a, a.conj()) - np.eye(a.shape[0]))) < 1e-12


def test_one_truncation_keeps_the_eckart_young_fraction():
    circ, p = W.config_c1(2)
    m, _ = M.run_circuit(circ, 32, canonical=True)
    g = W.haar_unitary(4, np.random.default_rng(9))
    q = 4
    exact = m.copy()
    M.apply_2q_canonical(exact, q, g, 32)
    trunc = m.copy()
    rec = M.apply_2q_canonical(trunc, q, g, 5, renormalize=False)
    assert rec.k == 5 and rec.eps > 1e-3
    a, b = M.to_dense(exact), M.to_dense(trunc)
    f = abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
    kept = np.sum(rec.s_all[:5] ** 2) / np.sum(rec.s_all ** 2)
    assert abs(f - kept) < 1e-12 and abs(np.vdot(b, b).real - kept) < 1e-12


def test_swap_chains_in_canonical_form_equal_dense():
    n = 8
    ops = W.nonlocal_ops(n, 40, 5)
    m, _ = M.run_ops(n, ops, 16, canonical=True)
    assert np.max(np.abs(M.to_dense(m) - D.run_ops(n, ops))) < 1e-12
