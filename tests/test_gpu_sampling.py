"""Perfect sampling on the GPU (tnsim_sample) against the oracle with the same uniforms.

Both sides draw b_q = 1 exactly when u[s, q] (p0 + p1) >= p0.  complex128 states
must give the oracle's bits exactly.  complex64 weights carry FP32 rounding, so a
shot may leave the oracle's path only at a draw whose uniform lies within 1e-4 of
the oracle's conditional probability p0 / (p0 + p1); every differing shot is
checked for that at its first differing qubit, and such shots must stay rare.
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


def _distinct_prefixes(bits):
    n = bits.shape[1]
    return sum(len({bytes(r[:q]) for r in bits}) for q in range(n))


def _conditional_p0(rc, nrm, prefix):
    """Oracle p0 / (p0 + p1) of the next qubit after ``prefix`` (right-canonical rc)."""
    v = np.ones((1,), np.complex128) / nrm
    for q, b in enumerate(prefix):
        w = v @ rc.sites[q][:, b, :]
        v = w / np.linalg.norm(w)
    a = rc.sites[len(prefix)]
    w0, w1 = v @ a[:, 0, :], v @ a[:, 1, :]
    p0, p1 = np.vdot(w0, w0).real, np.vdot(w1, w1).real
    return p0 / (p0 + p1)


def _check_against_oracle(bits, ref_bits, ref_mps, u, max_frac):
    diff = np.nonzero(np.any(bits != ref_bits, axis=1))[0]
    assert len(diff) <= max_frac * len(bits)
    if len(diff):
        rc = om.right_canonicalize(ref_mps)
        nrm = np.sqrt(om.norm2(rc))
        for s in diff:
            q = int(np.nonzero(bits[s] != ref_bits[s])[0][0])
            p0 = _conditional_p0(rc, nrm, ref_bits[s, :q])
            assert abs(u[s, q] - p0) < 1e-4, (s, q, u[s, q], p0)


@pytest.mark.parametrize("seed", [1, 2])
def test_complex128_bits_equal_the_oracle(T, seed):
    circ, p = W.config_c1(seed)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=p["chi_max"])
    m.run(circ)
    ref, _ = om.run_circuit(circ, p["chi_max"])
    u = np.random.default_rng(100 + seed).random((3000, 10))
    bits, nodes = T.tnsim_sample(m.h, u)
    assert np.array_equal(bits, om.perfect_sample_u(ref, u))
    assert nodes == _distinct_prefixes(bits)
    m.close()


def test_complex64_wide_state_against_the_oracle_on_its_own_sites(T):
    """60 qubits, chi_max 64, 14 brickwork layers: the oracle samples the GPU's
    exported state with the same uniforms."""
    n, chi = 60, 64
    circ = W.brickwork_su4(n, 14, 21)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi)
    m.run(circ)
    assert max(m.bond_dims()) == chi
    ref = om.MPS(m.export_sites())
    u = np.random.default_rng(7).random((600, n))
    bits, nodes = T.tnsim_sample(m.h, u)
    _check_against_oracle(bits, om.perfect_sample_u(ref, u), ref, u, 0.02)
    assert nodes == _distinct_prefixes(bits)
    m.close()


@pytest.mark.parametrize("dtype", ["C64", "C128"])
def test_ghz_closed_form(T, dtype):
    n = 40
    m = T.MPS(n, dtype=getattr(T, "TNSIM_" + dtype), chi_max=4)
    m.run(W.ghz_circuit(n))
    u = np.random.default_rng(3).random((500, n))
    bits, nodes = T.tnsim_sample(m.h, u)
    first = (u[:, 0] >= 0.5).astype(np.uint8)
    assert np.array_equal(bits, np.repeat(first[:, None], n, axis=1))
    assert nodes == 1 + 2 * (n - 1)        # two distinct prefixes at every length >= 1
    m.close()


def test_sampled_distribution_matches_born_rule(T):
    circ, p = W.config_c1(3)
    m = T.MPS(10, dtype=T.TNSIM_C64, chi_max=p["chi_max"])
    m.run(circ)
    probs = np.abs(dense.run_circuit(circ)) ** 2
    bits = m.sample(40000, seed=9)
    idx = bits.astype(np.int64) @ (1 << np.arange(9, -1, -1))
    emp = np.bincount(idx, minlength=1024) / len(idx)
    # sampling noise alone: E|f_i - p_i| <= sqrt(p_i (1 - p_i) / N), so the expected
    # total variation is at most half their sum (0.06 here); a biased sampler
    # (a wrong marginal anywhere) would add to it
    bound = 0.5 * np.sum(np.sqrt(probs * (1 - probs) / len(idx)))
    assert 0.5 * np.abs(emp - probs).sum() < 1.2 * bound
    m.close()


def test_rejects_uniforms_outside_the_unit_interval(T):
    m = T.MPS(4, dtype=T.TNSIM_C64, chi_max=4)
    for bad in (1.0, -0.1, np.nan):
        u = np.full((3, 4), 0.5)
        u[1, 2] = bad
        with pytest.raises(T.TnsimError) as ei:
            T.tnsim_sample(m.h, u)
        assert ei.value.status == T.TNSIM_EINVAL
    bits, nodes = T.tnsim_sample(m.h, np.zeros((0, 4)))
    assert bits.shape == (0, 4) and nodes == 0
    m.close()


@pytest.mark.slow
def test_full_size_chi256_state(T):
    """100 qubits with every interior bond at 256 (complex64, the bench's state):
    256 shots against the oracle sampling the exported sites."""
    n, chi = 100, 256
    circ = W.brickwork_su4(n, 12, 1000)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi)
    m.run(circ)
    assert max(m.bond_dims()) == chi
    ref = om.MPS(m.export_sites())
    u = np.random.default_rng(11).random((256, n))
    bits, _ = T.tnsim_sample(m.h, u)
    _check_against_oracle(bits, om.perfect_sample_u(ref, u), ref, u, 0.03)
    m.close()
