"""Pins of the oracle's perfect sampling with given uniforms (Sec. III.A "Sampling").

Shot s takes b_q = 1 exactly when u[s, q] * (p0 + p1) >= p0, with p0, p1 the
weights of the two outcomes of qubit q given the bits drawn before it.  Pinned by
* the chain rule computed directly on the dense vector |psi|^2 (marginals by
  summation over the undrawn qubits -- no MPS, no canonical form);
* closed forms: GHZ (all bits equal, decided by the first draw) and a product
  state (independent bits with p0 = |<0|phi_q>|^2).
"""
import numpy as np

import oracle.dense as D
import oracle.mps as M
import workloads as W


def _dense_chain_rule(psi, n, u):
    prob = np.abs(psi.reshape((2,) * n)) ** 2
    out = np.zeros((u.shape[0], n), np.uint8)
    for s in range(u.shape[0]):
        cond = prob
        for q in range(n):
            marg = cond.reshape(2, -1).sum(axis=1)      # weights of b_q = 0, 1
            b = 1 if u[s, q] * (marg[0] + marg[1]) >= marg[0] else 0
            cond = cond[b]
            out[s, q] = b
    return out


def test_sampling_follows_the_dense_chain_rule():
    rng = np.random.default_rng(5)
    for seed in (1, 2, 3):
        circ, p = W.config_c1(seed)
        mps, _ = M.run_circuit(circ, p["chi_max"])
        psi = D.run_circuit(circ)
        u = rng.random((300, circ.n_qubits))
        assert np.array_equal(M.perfect_sample_u(mps, u), _dense_chain_rule(psi, circ.n_qubits, u))


def test_sampling_ghz_closed_form():
    n = 12
    mps, _ = M.run_circuit(W.ghz_circuit(n), 4)
    u = np.random.default_rng(2).random((200, n))
    bits = M.perfect_sample_u(mps, u)
    first = (u[:, 0] >= 0.5).astype(np.uint8)
    assert np.array_equal(bits, np.repeat(first[:, None], n, axis=1))


def test_sampling_product_state_closed_form():
    n = 8
    rng = np.random.default_rng(4)
    us = [W.haar_unitary(2, rng) for _ in range(n)]
    mps = M.zero_state(n)
    for q in range(n):
        M.apply_1q(mps, q, us[q])
    p0 = np.array([abs(us[q][0, 0]) ** 2 for q in range(n)])
    u = rng.random((300, n))
    assert np.array_equal(M.perfect_sample_u(mps, u), (u >= p0[None, :]).astype(np.uint8))
