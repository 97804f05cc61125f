"""QR-preconditioned Jacobi SVD (bit 1 of tnsim_set_jacobi_config).

For a square gated block theta = Q R the Jacobi iteration runs on the columns of R^H,
the left site becomes theta V S^-1 and the right site S V^H is read off the converged
columns.  The kept spectra and the state must match the oracle layer by layer, the
left site must still be an isometry (the paper's form keeps U of Eq. 4), the
preconditioning must cut the Jacobi work, and states outside its scope (canonical
form) must run exactly as without it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mps as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    return T


def _isometry_err(site):
    """max |U^H U - I| of a site (chiL, 2, k) read as a (2 chiL) x k matrix."""
    u = site.reshape(-1, site.shape[2])
    return np.abs(u.conj().T @ u - np.eye(u.shape[1])).max()


def _check_layer(m, lay, chi, spec_tol, fid_tol, iso_tol):
    pre = om.MPS(m.export_sites())
    m.apply_layer(lay)
    sites = m.export_sites()
    for r in om.apply_layer(pre, lay, chi):
        sg = m.spectrum(r.q + 1)
        assert len(sg) == r.k and np.max(np.abs(sg - r.s_kept)) / r.s_kept[0] <= spec_tol
        assert _isometry_err(sites[r.q]) <= iso_tol
    assert 1 - om.fidelity(om.MPS(sites), pre) <= fid_tol


@pytest.mark.parametrize("cfg", [2, 3])
def test_qr_layers_complex128(T, cfg):
    """16 qubits, chi 32, every layer truncating: spectra, state and left isometries
    against the oracle in complex128."""
    circ = W.brickwork_u2_su4(16, 10, seed=21)
    m = T.MPS(16, dtype=T.TNSIM_C128, chi_max=32)
    T.tnsim_set_jacobi_config(m.h, cfg)
    for lay in circ.layers:
        _check_layer(m, lay, 32, 1e-10, 1e-12, 1e-10)
    m.close()


@pytest.mark.parametrize("cfg", [2, 6])
def test_qr_saturated_layers_complex64(T, cfg):
    """40 qubits at chi 128 (square 256 x 256 gated blocks in the bulk), complex64,
    tensor-core contraction: the layers after the bond dimension saturates (with the
    column rotations, and with the Gram-matrix visits on the tensor cores)."""
    n = 40
    circ = W.brickwork_su4(n, 11, seed=5)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=128, gemm=T.TNSIM_GEMM_TF32X3)
    m.run(W.Circuit(n, circ.layers[:8]))
    T.tnsim_set_jacobi_config(m.h, cfg)
    for lay in circ.layers[8:]:
        _check_layer(m, lay, 128, 1e-5, 1e-6, 1e-4)
    m.close()


def test_qr_cuts_the_jacobi_work(T):
    """The same saturated layer from the same state: fewer examined column pairs with
    the preconditioning, the same kept bond dimensions."""
    n = 40
    circ = W.brickwork_su4(n, 9, seed=5)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=128)
    m.run(W.Circuit(n, circ.layers[:8]))
    sites = m.export_sites()
    lay = circ.layers[8]
    work = {}
    for cfg in (0, 2):
        s = T.MPS(n, dtype=T.TNSIM_C64, chi_max=128)
        s.import_sites(sites)
        T.tnsim_set_jacobi_config(s.h, cfg)
        T.tnsim_last_stats(s.h)
        s.apply_layer(lay)
        work[cfg] = (T.tnsim_last_stats(s.h), list(s.bond_dims()))
        s.close()
    (plain, dims0), (pre, dims2) = work[0], work[2]
    assert dims0 == dims2
    assert pre["gates"] == plain["gates"]
    assert pre["visit_rows"] < 0.9 * plain["visit_rows"]
    # the Householder count 2 n^3 / 3 of every preconditioned gate, none without
    assert plain["qr_cmacs"] == 0 and pre["qr_cmacs"] > 0
    m.close()


@pytest.mark.parametrize("dt,fid_tol", [("C128", 1e-12), ("C64", 1e-6)])
def test_qr_in_a_replayed_plan(T, dt, fid_tol):
    """A frozen layer plan of a state that selected the preconditioning gives the
    layer-by-layer result."""
    dtype = getattr(T, "TNSIM_" + dt)
    circ = W.brickwork_u2_su4(14, 6, seed=13)
    ref = T.MPS(14, dtype=dtype, chi_max=16)
    T.tnsim_set_jacobi_config(ref.h, 2)
    ref.run(circ)
    want = ref.export_sites()
    torch = pytest.importorskip("torch")
    m = T.MPS(14, dtype=dtype, chi_max=16)
    T.tnsim_set_jacobi_config(m.h, 2)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()

    bufs = [(dev(l.g4), dev(l.u1)) for l in circ.layers]
    torch.cuda.synchronize()
    plans = [T.tnsim_plan_create([m.h], [(l.pairs, g.data_ptr(), u.data_ptr())])
             for l, (g, u) in zip(circ.layers, bufs)]
    for p in plans:
        T.tnsim_plan_launch(p)
    m.sync()
    got = m.export_sites()
    assert 1 - om.fidelity(om.MPS(got), om.MPS(want)) <= fid_tol
    for p in plans:
        T.tnsim_plan_destroy(p)
    m.close()
    ref.close()


def test_canonical_form_ignores_the_preconditioning(T):
    """Canonical-form gates never take the QR path: configurations 0 and 2 run the
    same kernels on the same data and give identical sites."""
    circ = W.brickwork_u2_su4(12, 6, seed=2)
    out = []
    for cfg in (0, 2):
        m = T.MPS(12, dtype=T.TNSIM_C64, chi_max=16, form=T.TNSIM_FORM_CANONICAL)
        T.tnsim_set_jacobi_config(m.h, cfg)
        m.run(circ)
        out.append(m.export_sites())
        m.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
