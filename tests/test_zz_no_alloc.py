"""tnsim_two_site_update_noalloc against tnsim_apply_layer and the FP64 oracle.

The no-allocation entry point exists for callers that may not let the library call
cudaMalloc (a plugin inside an application whose memory pool owns the device, a
fixed device-memory budget, a loop that must not synchronise the device).  It works
in a fixed scratch array compiled into the library, so this test checks that two
calls in a row -- the second one smaller than the first, on the leftovers of the
first -- give the same update as the ordinary handle-based path, within the
complex64 tolerances of the other GPU tests (singular values within 1e-5 of s_max,
the gauge-invariant two-site block within 1e-5 relative), and the update of the
oracle (oracle.mps.apply_2q on the same complex64-rounded sites): singular values
within 1e-5 of s_max, the discarded weight within 1e-6, and the two-site block at
1 - F <= 1e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sites(n, chi, seed):
    rng = np.random.default_rng(seed)
    d = [min(2 ** b, 2 ** (n - b), chi) for b in range(n + 1)]
    return [((rng.standard_normal((d[i], 2, d[i + 1])) + 1j * rng.standard_normal((d[i], 2, d[i + 1])))
             / np.sqrt(2 * d[i + 1])) for i in range(n)], d


def test_noalloc_update_matches_layer_path_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    import workloads as W
    from oracle import mps as om

    n, q = 16, 7
    for call, (chi, chi_max, seed) in enumerate(((128, 128, 11), (32, 32, 12))):
        sites, d = _sites(n, chi, seed)
        gate = W.haar_su4(np.random.default_rng(100 + call))
        cl, cm, cr = d[q], d[q + 1], d[q + 2]

        # the existing entry point
        m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi_max)
        m.import_sites([s.astype(np.complex64).astype(np.complex128) for s in sites])
        eps_ref = T.tnsim_apply_layer(m.h, np.array([q], np.int32), gate[None])[0]
        s_ref = m.spectrum(q + 1)
        out = m.export_sites()
        m.close()

        # the no-allocation entry point on caller-owned device buffers
        kmax = min(chi_max, 2 * cl, 2 * cr)
        bond = max(cm, kmax)
        cap_a, cap_b = cl * 2 * bond, bond * 2 * cr
        A = torch.zeros(cap_a, dtype=torch.complex64, device="cuda")
        B = torch.zeros(cap_b, dtype=torch.complex64, device="cuda")
        A[: cl * 2 * cm].copy_(torch.from_numpy(sites[q].astype(np.complex64).reshape(-1)))
        B[: cm * 2 * cr].copy_(torch.from_numpy(sites[q + 1].astype(np.complex64).reshape(-1)))
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        k, eps, s = T.tnsim_two_site_update_noalloc(A.data_ptr(), cap_a, B.data_ptr(), cap_b, cl, cm, cr,
                                                   gate, chi_max, 0.0, True, stream=stream.cuda_stream)
        torch.cuda.synchronize()

        assert k == len(s_ref) == out[q].shape[2]
        assert np.max(np.abs(s - s_ref)) / s_ref[0] <= 1e-5
        assert abs(eps - eps_ref) <= 1e-5
        a_new = A[: cl * 2 * k].cpu().numpy().astype(np.complex128).reshape(cl, 2, k)
        b_new = B[: k * 2 * cr].cpu().numpy().astype(np.complex128).reshape(k, 2, cr)
        blk = np.einsum("lxb,byr->lxyr", a_new, b_new)
        blk_ref = np.einsum("lxb,byr->lxyr", out[q], out[q + 1])
        assert np.linalg.norm(blk - blk_ref) / np.linalg.norm(blk_ref) <= 1e-5

        # the oracle's update of the same complex64-rounded sites
        ref = om.MPS([s_.astype(np.complex64).astype(np.complex128) for s_ in sites])
        rec = om.apply_2q(ref, q, gate, chi_max)
        assert k == rec.k
        assert np.max(np.abs(s - rec.s_kept)) / rec.s_kept[0] <= 1e-5
        assert abs(eps - rec.eps) <= 1e-6
        blk_o = np.einsum("lxb,byr->lxyr", ref.sites[q], ref.sites[q + 1])
        f = abs(np.vdot(blk_o, blk)) ** 2 / (np.vdot(blk_o, blk_o).real * np.vdot(blk, blk).real)
        assert 1.0 - f <= 1e-6


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T

    A = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TnsimError) as ei:
        T.tnsim_two_site_update_noalloc(A.data_ptr(), 1 << 20, A.data_ptr(), 1 << 20, 129, 4, 4,
                                        np.eye(4), 64)
    assert ei.value.status == T.TNSIM_EINVAL and "128" in str(ei.value)
