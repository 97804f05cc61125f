"""Non-local two-qubit gates (Sec. IV.B SWAP method) and layerization, on the CPU.

* the dense any-pair gate (the plain contraction of Eq. 1 on two arbitrary legs)
  against a brute-force sum over basis states and against the closed form of CX;
* the oracle's SWAP chain against that dense contraction, untruncated;
* SWAP applied twice is the identity, and a truncating SWAP chain respects chi_max;
* the library's host planner (tnsim_circuit_layerize: no GPU work) -- disjoint
  pairs per layer, the SWAP count, its layers replayed by the dense oracle equal
  the gate list applied in order, and its argument checks.
"""
import numpy as np
import pytest

import oracle.dense as D
import oracle.mps as M
import workloads as W


def _brute_any(psi, n, qa, qb, g):
    """psi'[i] = sum_j G[(2 a_i + b_i), (2 a_j + b_j)] psi[j] over all j that agree with i
    on every other qubit (qubit 0 = most significant bit)."""
    out = np.zeros_like(psi)
    bit = lambda x, q: (x >> (n - 1 - q)) & 1
    for i in range(2 ** n):
        for j in range(2 ** n):
            if any(bit(i, k) != bit(j, k) for k in range(n) if k not in (qa, qb)):
                continue
            out[i] += g[2 * bit(i, qa) + bit(i, qb), 2 * bit(j, qa) + bit(j, qb)] * psi[j]
    return out


def test_dense_any_pair_matches_brute_force():
    rng = np.random.default_rng(3)
    n = 4
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    for qa in range(n):
        for qb in range(n):
            if qa == qb:
                continue
            g = W.haar_unitary(4, rng)
            assert np.allclose(D.apply_2q_any(psi, n, qa, qb, g), _brute_any(psi, n, qa, qb, g), atol=1e-13)


def test_dense_any_pair_cx_closed_form():
    n = 5
    cx = W.gate_cx()          # control = first listed qubit
    for qa, qb in ((0, 4), (4, 0), (1, 3), (3, 2)):
        for x in range(2 ** n):
            psi = np.zeros(2 ** n, np.complex128)
            psi[x] = 1.0
            out = D.apply_2q_any(psi, n, qa, qb, cx)
            ctrl = (x >> (n - 1 - qa)) & 1
            y = x ^ (ctrl << (n - 1 - qb))
            assert out[y] == 1.0 and np.count_nonzero(out) == 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_swap_chain_equals_dense(seed):
    n = 8
    ops = W.nonlocal_ops(n, 40, seed)
    m, recs = M.run_ops(n, ops, chi_max=16)     # 2^(n/2): nothing is truncated
    psi = D.run_ops(n, ops)
    assert np.max(np.abs(M.to_dense(m) - psi)) < 1e-12
    n_two = sum(1 for _, b, _ in ops if b is not None)
    n_swaps = sum(2 * (abs(a - b) - 1) for a, b, _ in ops if b is not None)
    assert len(recs) == n_two + n_swaps


def test_oracle_swap_twice_is_identity_and_truncation_caps_bonds():
    n = 10
    m0, _ = M.run_ops(n, W.nonlocal_ops(n, 30, 7, max_dist=1), chi_max=32)
    m = m0.copy()
    M.apply_2q(m, 4, M.SWAP, 32)
    M.apply_2q(m, 4, M.SWAP, 32)
    assert 1.0 - M.fidelity(m, m0) < 1e-12
    # a truncating chain: every bond within chi_max, and some weight was discarded
    mt, recs = M.run_ops(n, W.nonlocal_ops(n, 30, 8), chi_max=4)
    assert max(mt.bond_dims()) <= 4 and max(r.eps for r in recs) > 0.0


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    return T


def _replay_dense(n, layers):
    psi = D.zero_state(n)
    for q, g4, u1 in layers:
        for x in range(n):
            psi = D.apply_1q(psi, n, x, u1[x])
        for qq, g in zip(q, g4):
            psi = D.apply_2q(psi, n, int(qq), g)
    return psi


@pytest.mark.parametrize("seed,max_dist", [(1, None), (2, 2), (3, 1)])
def test_planner_layers_replay_to_the_gate_list(T, seed, max_dist):
    n = 9
    ops = W.nonlocal_ops(n, 50, seed, p1=0.3, max_dist=max_dist)
    layers = T.tnsim_circuit_layerize(n, ops)
    for q, _, _ in layers:
        used = np.concatenate([q, q + 1])
        assert len(set(used.tolist())) == len(used) and np.all(q >= 0) and np.all(q < n - 1)
    n_local = sum(len(q) for q, _, _ in layers)
    assert n_local == sum(2 * abs(a - b) - 1 for a, b, _ in ops if b is not None)
    assert np.max(np.abs(_replay_dense(n, layers) - D.run_ops(n, ops))) < 1e-12
    # as-soon-as-possible: no more layers than local operations in sequence
    assert len(layers) <= n_local + sum(1 for _, b, _ in ops if b is None)


def test_planner_packs_independent_gates_into_one_layer(T):
    n = 8
    ops = [(0, 1, np.eye(4)), (2, 3, np.eye(4)), (5, 4, np.eye(4)), (6, 7, np.eye(4)), (3, None, np.eye(2))]
    layers = T.tnsim_circuit_layerize(n, ops)
    assert len(layers) == 2 and sorted(layers[0][0].tolist()) == [0, 2, 4, 6]


def test_planner_rejects_bad_operations(T):
    g = np.eye(4)
    for ops in ([(2, 2, g)], [(0, 9, g)], [(-1, 3, g)], [(1, 2, np.full((4, 4), np.nan))]):
        with pytest.raises(T.TnsimError) as ei:
            T.tnsim_circuit_layerize(8, ops)
        assert ei.value.status == T.TNSIM_EINVAL
    assert T.tnsim_circuit_layerize(8, []) == []
