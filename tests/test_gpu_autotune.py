"""The Jacobi launch configurations and their autotuner (tnsim_autotune).

Every configuration must give the oracle's results (they change the block width,
hence the order of the rotations, and whether the Jacobi iteration runs on theta or
on R^H of its QR factorisation); the autotuner must leave the state exactly as it
was and pick one of them.
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


@pytest.mark.parametrize("cfg", range(8))
def test_every_configuration_exact_complex128(T, cfg):
    circ, p = W.config_c1(2)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=p["chi_max"])
    T.tnsim_set_jacobi_config(m.h, cfg)
    m.run(circ)
    psi = dense.run_circuit(circ)
    amps = m.amplitudes(_all_bits(10))
    assert np.linalg.norm(amps - psi) / np.linalg.norm(psi) < 1e-10
    m.close()


@pytest.mark.parametrize("cfg", range(8))
def test_every_configuration_exact_complex128_wide_blocks(T, cfg):
    """14 qubits without truncation (bonds up to 128, gated blocks up to 256 rows,
    several column blocks per gate in every configuration): the dense state vector
    within 1e-10."""
    n = 14
    circ = W.brickwork_su4(n, 12, seed=8)
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=128)
    T.tnsim_set_jacobi_config(m.h, cfg)
    m.run(circ)
    assert max(m.bond_dims()) == 128
    psi = dense.run_circuit(circ)
    amps = m.amplitudes(_all_bits(n))
    assert np.linalg.norm(amps - psi) / np.linalg.norm(psi) < 1e-10
    m.close()


@pytest.mark.parametrize("cfg", range(8))
def test_every_configuration_complex64_per_layer(T, cfg):
    """24 qubits, chi 64 (m up to 128): every layer against the oracle on the same input."""
    circ = W.brickwork_u2_su4(24, 9, seed=6)
    m = T.MPS(24, dtype=T.TNSIM_C64, chi_max=64)
    T.tnsim_set_jacobi_config(m.h, cfg)
    for lay in circ.layers:
        pre = om.MPS(m.export_sites())
        m.apply_layer(lay)
        for r in om.apply_layer(pre, lay, 64):
            sg = m.spectrum(r.q + 1)
            assert len(sg) == r.k and np.max(np.abs(sg - r.s_kept)) / r.s_kept[0] <= 1e-5
        assert 1 - om.fidelity(om.MPS(m.export_sites()), pre) <= 1e-6
    m.close()


def test_autotune_keeps_the_state_and_picks_a_configuration(T):
    n = 40
    circ = W.brickwork_su4(n, 10, seed=3)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=128)
    m.run(W.Circuit(n, circ.layers[:8]))
    before = m.export_sites()
    dims = list(m.bond_dims())
    lay = circ.layers[8]
    choice, ms = T.tnsim_autotune(m.h, lay.pairs, lay.g4, reps=2)
    assert choice in range(T.TNSIM_JACOBI_CONFIGS) and len(ms) == T.TNSIM_JACOBI_CONFIGS and np.all(ms > 0) and ms[choice] == ms.min()
    assert list(m.bond_dims()) == dims
    for a, b in zip(m.export_sites(), before):
        assert np.array_equal(a, b)
    # the next layer runs in the chosen configuration and still matches the oracle
    pre = om.MPS(before)
    m.apply_layer(lay)
    for r in om.apply_layer(pre, lay, 128):
        sg = m.spectrum(r.q + 1)
        assert len(sg) == r.k and np.max(np.abs(sg - r.s_kept)) / r.s_kept[0] <= 1e-5
    with pytest.raises(T.TnsimError):
        T.tnsim_set_jacobi_config(m.h, T.TNSIM_JACOBI_CONFIGS)
    m.close()
