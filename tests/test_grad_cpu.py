"""Pins of the oracle's reverse-mode energy gradient (oracle/grad.py).

* the truncation backward returns exactly Pb for a loss of the product P = U Y alone
  (also with degenerate singular values, where the textbook 1/(s_i^2 - s_j^2)
  formula breaks down);
* the final-state adjoint against finite differences of the energy in each site entry;
* the whole gradient against central finite differences of the energy computed by
  the dense state-vector simulator (untruncated), and of the oracle's own truncated
  simulation (chi_max below the exact rank), where it is the exact derivative;
* the rotation convention R_a(t) = exp(-i t P_a / 2) against the closed forms used
  by the circuit generator.
"""
import numpy as np
import pytest

import oracle.dense as D
import oracle.grad as G
import oracle.mps as M
import workloads as W


def _haar(rng, d):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("svals", [[1.0, 0.8, 0.5, 0.3], [1.0, 1.0, 0.3, 0.3], [0.7, 0.7, 0.7, 0.7]])
def test_truncation_backward_of_a_product_loss_is_its_adjoint(svals):
    rng = np.random.default_rng(0)
    m, n = 4, 8
    T = _haar(rng, m) @ np.diag(svals) @ _haar(rng, n)[:, :4].conj().T
    u, s, _ = np.linalg.svd(T, full_matrices=False)
    Y = u.conj().T @ T
    Pb = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    tb = G.truncation_backward(T, u, Y, s, 4, u, Pb @ Y.conj().T, u.conj().T @ Pb)
    assert np.max(np.abs(tb - Pb)) < 1e-12


def test_final_adjoint_against_finite_differences():
    n = 5
    m, _ = M.run_circuit(W.brickwork_u2_su4(n, 3, seed=2), 8)
    paulis, coeffs = ["ZZIII", "IZZII", "XIIII", "IIIXI", "IYYII"], [1.0, 0.7, 0.5, 0.3, -0.4]
    e, ab = G.final_adjoint(m, paulis, coeffs)
    assert abs(e - G.energy(m, paulis, coeffs)) < 1e-13
    h = 1e-6
    for q in range(n):
        for idx in [(0, 0, 0), tuple(x - 1 for x in m.sites[q].shape)]:
            for d in (1.0, 1j):
                mp, mm = m.copy(), m.copy()
                mp.sites[q] = m.sites[q].copy(); mp.sites[q][idx] += h * d
                mm.sites[q] = m.sites[q].copy(); mm.sites[q][idx] -= h * d
                fd = (G.energy(mp, paulis, coeffs) - G.energy(mm, paulis, coeffs)) / (2 * h)
                assert abs(fd - 2 * np.real(np.conj(ab[q][idx]) * d)) < 1e-8


def _hea(n, n_layers, seed, sigma=0.5):
    circ, angles = W.hea_circuit(n, n_layers, seed=seed, sigma=sigma)
    layers = [(l.pairs, l.g4) for l in circ.layers]
    axes = ["YZ" if i % 2 == 0 else "" for i in range(len(layers))]
    theta = [angles[i // 2].copy() if i % 2 == 0 else np.zeros((n, 0)) for i in range(len(layers))]
    paulis = ["".join("Z" if k in (i, i + 1) else "I" for k in range(n)) for i in range(n - 1)] + \
             ["".join("X" if k == i else "I" for k in range(n)) for i in range(n)]
    coeffs = [1.0] * (n - 1) + [0.5] * n
    return layers, axes, theta, paulis, coeffs


def _dense_energy(n, layers, axes, theta, paulis, coeffs):
    psi = D.zero_state(n)
    for L, (pairs, g4) in enumerate(layers):
        u1 = G.layer_u1(n, axes[L], theta[L])
        if u1 is not None:
            for q in range(n):
                psi = D.apply_1q(psi, n, q, u1[q])
        for q, g in zip(pairs, g4):
            psi = D.apply_2q(psi, n, int(q), g)
    return sum(c * D.expect_pauli(psi, n, p).real for p, c in zip(paulis, coeffs)) / np.vdot(psi, psi).real


def _fd_check(grads, theta, energy_fn, tol, h=1e-6):
    worst = 0.0
    for L, t in enumerate(theta):
        for idx in np.ndindex(t.shape):
            tp = [x.copy() for x in theta]; tm = [x.copy() for x in theta]
            tp[L][idx] += h; tm[L][idx] -= h
            fd = (energy_fn(tp) - energy_fn(tm)) / (2 * h)
            worst = max(worst, abs(fd - grads[L][idx]))
    assert worst < tol, worst


def test_gradient_untruncated_against_dense_finite_differences():
    n = 6
    layers, axes, theta, paulis, coeffs = _hea(n, 3, seed=3)
    e, grads = G.grad(n, layers, axes, theta, paulis, coeffs, chi_max=64)
    assert abs(e - _dense_energy(n, layers, axes, theta, paulis, coeffs)) < 1e-12
    _fd_check(grads, theta, lambda th: _dense_energy(n, layers, axes, th, paulis, coeffs), 1e-7)


@pytest.mark.parametrize("chi", [2, 3, 4])
def test_gradient_truncated_against_the_oracles_own_finite_differences(chi):
    n = 6
    layers, axes, theta, paulis, coeffs = _hea(n, 3, seed=3)

    def en(th):
        m, _ = G.run(n, layers, axes, th, chi)
        return G.energy(m, paulis, coeffs)

    e, grads = G.grad(n, layers, axes, theta, paulis, coeffs, chi_max=chi)
    assert abs(e - en(theta)) < 1e-13
    _fd_check(grads, theta, en, 1e-7)


def test_rotation_convention():
    for t in (0.3, -1.1, 2.0):
        assert np.allclose(G.rotation("X", t), W.gate_rx(t), atol=1e-15)
        assert np.allclose(G.rotation("Y", t), W.gate_ry(t), atol=1e-15)
        assert np.allclose(G.rotation("Z", t), W.gate_rz(t), atol=1e-15)


def test_energy_local_equals_full_transfer():
    """energy_local (each string contracted over its support between identity
    environments) equals the full-chain energy on a random, unnormalised MPS."""
    rng = np.random.default_rng(31)
    n = 7
    dims = [1, 2, 4, 5, 5, 4, 2, 1]
    sites = [rng.standard_normal((dims[q], 2, dims[q + 1])) + 1j * rng.standard_normal((dims[q], 2, dims[q + 1]))
             for q in range(n)]
    m = M.MPS(sites)
    paulis = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(12)]
    paulis += ["I" * n, "Z" + "I" * (n - 1), "I" * (n - 1) + "X", "IIZZIII", "XIIIIIY"]
    coeffs = rng.standard_normal(len(paulis))
    assert abs(G.energy_local(m, paulis, coeffs) - G.energy(m, paulis, coeffs)) < 1e-12 * max(
        1.0, abs(G.energy(m, paulis, coeffs)))
