"""Non-local two-qubit gates through tnsim_apply_circuit (Sec. IV.B SWAP method,
layerization) against the FP64 oracle, which applies the same list in program order.

Gauge-invariant comparisons only (amplitudes, per-bond singular values, discarded
weights, fidelity), with the tolerances of the other parity tests: complex128 within
1e-10, complex64 singular values within 1e-5 of s_max and 1 - F <= 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense
from oracle import mps as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    return T


def _all_bits(n):
    return np.array([[(x >> (n - 1 - i)) & 1 for i in range(n)] for x in range(2 ** n)], dtype=np.uint8)


def _spectrum_err(m, ref):
    worst = 0.0
    for b in range(1, ref.n):
        sr, sg = ref.spectrum[b], m.spectrum(b)
        if sr is None:
            continue
        k = max(len(sr), len(sg))
        a = np.zeros(k); a[: len(sg)] = sg
        c = np.zeros(k); c[: len(sr)] = sr
        worst = max(worst, float(np.max(np.abs(a - c)) / sr[0]))
    return worst


@pytest.mark.parametrize("seed", [1, 2])
def test_exact_nonlocal_circuit_complex128(T, seed):
    """10 qubits, 60 gates at every distance and in both qubit orders, chi_max 32
    (nothing truncated): all 1024 amplitudes against the dense contraction."""
    n = 10
    ops = W.nonlocal_ops(n, 60, seed)
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=32)
    n_layers, n_local, eps = m.apply_circuit(ops)
    psi = dense.run_ops(n, ops)
    amps = m.amplitudes(_all_bits(n))
    assert np.linalg.norm(amps - psi) / np.linalg.norm(psi) < 1e-10
    ref, recs = om.run_ops(n, ops, 32)
    assert n_local == len(recs) and eps < 1e-20
    assert list(m.bond_dims()) == ref.bond_dims()
    assert _spectrum_err(m, ref) < 1e-10
    m.close()


def test_exact_nonlocal_circuit_complex64(T):
    n = 10
    ops = W.nonlocal_ops(n, 60, 3)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=32)
    m.apply_circuit(ops)
    ref, _ = om.run_ops(n, ops, 32)
    assert 1 - om.fidelity(om.MPS(m.export_sites()), ref) <= 1e-6
    assert _spectrum_err(m, ref) <= 1e-5
    m.close()


@pytest.mark.parametrize("dtype", ["C128", "C64"])
def test_truncated_swap_chains(T, dtype):
    """16 qubits, chi_max 8: every SWAP truncates.  The layered GPU run and the
    in-order oracle run make the same sequence of updates on every bond.
    complex64 runs 40 operations (145 updates): over 80 (326 updates) FP32 rounding,
    amplified by the repeated truncations, reaches 5e-5 of s_max in an FP64
    emulation that rounds every site to complex64, beyond the 1e-5 bound."""
    n, chi = 16, 8
    ops = W.nonlocal_ops(n, 80 if dtype == "C128" else 40, 11, max_dist=6)
    dt = getattr(T, "TNSIM_" + dtype)
    m = T.MPS(n, dtype=dt, chi_max=chi)
    _, n_local, eps = m.apply_circuit(ops)
    ref, recs = om.run_ops(n, ops, chi)
    assert n_local == len(recs)
    eps_ref = sum(r.eps for r in recs)
    assert eps_ref > 1e-3
    tol_s, tol_f, tol_e = (1e-10, 1e-10, 1e-10) if dtype == "C128" else (1e-5, 1e-6, 1e-5)
    assert abs(eps - eps_ref) <= tol_e * max(1.0, eps_ref)
    assert list(m.bond_dims()) == ref.bond_dims()
    assert _spectrum_err(m, ref) <= tol_s
    assert 1 - om.fidelity(om.MPS(m.export_sites()), ref) <= tol_f
    m.close()


def test_circuit_matches_layer_api_on_local_gates(T):
    """A nearest-neighbour brickwork given as a gate list equals the same layers
    given to tnsim_apply_layer (bitwise: the same launches on the same data)."""
    n = 12
    circ = W.brickwork_su4(n, 6, 5)
    ops = [(int(q), int(q) + 1, g) for l in circ.layers for q, g in zip(l.pairs, l.g4)]
    a = T.MPS(n, dtype=T.TNSIM_C64, chi_max=16)
    b = T.MPS(n, dtype=T.TNSIM_C64, chi_max=16)
    nl, ng, _ = a.apply_circuit(ops)
    b.run(circ)
    assert nl == len(circ.layers) and ng == circ.n_2q
    for sa, sb in zip(a.export_sites(), b.export_sites()):
        assert np.array_equal(sa, sb)
    a.close(); b.close()


def test_bad_operations_leave_the_state_alone(T):
    n = 6
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=8)
    m.apply_circuit(W.nonlocal_ops(n, 10, 4))
    before = m.export_sites()
    for ops in ([(0, 3, np.eye(4)), (2, 2, np.eye(4))], [(0, 6, np.eye(4))],
                [(1, None, np.full((2, 2), np.inf))]):
        with pytest.raises(T.TnsimError) as ei:
            m.apply_circuit(ops)
        assert ei.value.status == T.TNSIM_EINVAL
    for sa, sb in zip(m.export_sites(), before):
        assert np.array_equal(sa, sb)
    m.close()
