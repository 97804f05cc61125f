"""Canonical-form two-qubit updates (TNSIM_FORM_CANONICAL, Hastings form) against
the oracle's apply_2q_canonical.

Gauge-invariant comparisons as in the other parity tests (amplitudes, bond spectra,
discarded weights, fidelity; complex128 within 1e-10, complex64 singular values
within 1e-5 of s_max and 1 - F <= 1e-6), plus the properties the form promises:
the stored spectra are the Schmidt coefficients of the state, and every site right
of the first is a right isometry (untruncated runs).
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


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_complex128_schmidt_spectra_and_isometries(T, seed):
    circ, p = W.config_c1(seed)
    n = circ.n_qubits
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=p["chi_max"], form=T.TNSIM_FORM_CANONICAL)
    m.run(circ)
    psi = dense.run_circuit(circ)
    amps = m.amplitudes(_all_bits(n))
    assert np.linalg.norm(amps - psi) / np.linalg.norm(psi) < 1e-10
    for b in range(1, n):
        sv = np.linalg.svd(psi.reshape(2 ** b, -1), compute_uv=False)
        lam = m.spectrum(b)
        assert np.max(np.abs(sv[: len(lam)] - lam)) < 1e-10
    for a in m.export_sites()[1:]:
        assert np.max(np.abs(np.einsum("lpr,mpr->lm", a, a.conj()) - np.eye(a.shape[0]))) < 1e-10
    m.close()


@pytest.mark.parametrize("dtype,depth", [("C128", 14), ("C64", 6)])
def test_truncated_brickwork_against_the_canonical_oracle(T, dtype, depth):
    n, chi = 24, 16
    circ = W.brickwork_u2_su4(n, depth, 31)
    m = T.MPS(n, dtype=getattr(T, "TNSIM_" + dtype), chi_max=chi, form=T.TNSIM_FORM_CANONICAL)
    eps = m.run(circ)
    ref, recs = om.run_circuit(circ, chi, canonical=True)
    eps_ref = [np.array([r.eps for r in layer]) for layer in recs]
    assert max(float(np.max(e)) for e in eps_ref if len(e)) > 1e-4
    tol_s, tol_f = (1e-10, 1e-10) if dtype == "C128" else (1e-5, 1e-6)
    for e, er in zip(eps, eps_ref):
        assert np.max(np.abs(e - er), initial=0.0) <= tol_s
    assert list(m.bond_dims()) == ref.bond_dims()
    assert _spectrum_err(m, ref) <= tol_s
    assert 1 - om.fidelity(om.MPS(m.export_sites()), ref) <= tol_f
    m.close()


@pytest.mark.parametrize("gemm", ["FP32", "FP32_3M", "TF32X3", "BF16X3"])
def test_canonical_form_with_every_contraction_mode(T, gemm):
    """Every complex64 contraction mode, layer by layer: the canonical oracle applied
    to the GPU's own input state (its sites and bond spectra) against the GPU's
    result -- singular values within 1e-5 of s_max, 1 - F <= 1e-6 per layer."""
    n, chi = 16, 8
    circ = W.brickwork_u2_su4(n, 8, 8)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi, form=T.TNSIM_FORM_CANONICAL,
              gemm=getattr(T, "TNSIM_GEMM_" + gemm))
    for lay in circ.layers:
        pre = om.MPS(m.export_sites())
        for b in range(1, n):
            sp = m.spectrum(b)
            pre.spectrum[b] = sp if len(sp) else None
        m.apply_layer(lay)
        for r in om.apply_layer(pre, lay, chi, canonical=True):
            sg = m.spectrum(r.q + 1)
            assert len(sg) == r.k
            assert np.max(np.abs(sg - r.s_kept)) / r.s_kept[0] <= 1e-5
        assert 1 - om.fidelity(om.MPS(m.export_sites()), pre) <= 1e-6
    m.close()


def test_canonical_swap_chains(T):
    n, chi = 14, 8
    ops = W.nonlocal_ops(n, 40, 12, max_dist=5)
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=chi, form=T.TNSIM_FORM_CANONICAL)
    _, n_local, eps = m.apply_circuit(ops)
    ref, recs = om.run_ops(n, ops, chi, canonical=True)
    assert n_local == len(recs) and abs(eps - sum(r.eps for r in recs)) < 1e-10
    assert _spectrum_err(m, ref) < 1e-10
    assert 1 - om.fidelity(om.MPS(m.export_sites()), ref) < 1e-10
    m.close()


def test_canonical_truncation_beats_the_papers_form(T):
    """The point of the form: at the same chi_max the state stays closer to the exact one."""
    n = 16
    circ = W.brickwork_su4(n, 12, 3)
    psi = dense.run_circuit(circ)
    bits = _all_bits(n)
    fid = {}
    for form in ("PAPER", "CANONICAL"):
        m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=16, form=getattr(T, "TNSIM_FORM_" + form))
        m.run(circ)
        a = m.amplitudes(bits)
        fid[form] = abs(np.vdot(a, psi)) ** 2 / (np.vdot(a, a).real * np.vdot(psi, psi).real)
        m.close()
    assert fid["CANONICAL"] > fid["PAPER"] + 0.1


def test_import_into_a_canonical_state_is_refused(T):
    m = T.MPS(6, dtype=T.TNSIM_C64, chi_max=4, form=T.TNSIM_FORM_CANONICAL)
    sites = m.export_sites()
    with pytest.raises(T.TnsimError) as ei:
        m.import_sites(sites)
    assert ei.value.status == T.TNSIM_EUNSUPPORTED
    m.close()
