"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

The SVD gauge is not unique, so only gauge-invariant quantities are compared:
amplitudes <x|psi> (phase included), per-bond singular values, discarded weights,
bond dimensions, Pauli expectations and the state fidelity
F = |<a|b>|^2 / (<a|a><b|b>).  Tolerances:
  complex128 runs: 1e-10 relative;
  complex64 runs: singular values within 1e-5 of s_max per bond (normwise) and
  1 - F <= 1e-6; amplitude and expectation bounds are derived from F
  (|a_gpu - a_ref| / |a_ref| <= 2 sqrt(1 - F) on a set of strings, which gives 2e-3).
  Over many truncated layers complex64 is compared layer by layer (see the C2 tests).
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


def _fidelity(sites_a, sites_b):
    return om.fidelity(om.MPS(sites_a), om.MPS(sites_b))


def _spectrum_err(m, ref, chi_max):
    """max over bonds of max_j |s_gpu - s_ref| / s_max (zero-padded)."""
    worst = 0.0
    for b in range(1, ref.n):
        sr = ref.spectrum[b]
        sg = m.spectrum(b)
        if sr is None:
            assert len(sg) == 0
            continue
        k = max(len(sr), len(sg))
        a = np.zeros(k); a[: len(sg)] = sg
        c = np.zeros(k); c[: len(sr)] = sr
        worst = max(worst, float(np.max(np.abs(a - c)) / sr[0]))
    return worst


# ----------------------------------------------------------------- complex128, exact


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_c1_complex128_exact(T, seed):
    """10 qubits, depth 8, U(2) + SU(4), chi_max 32 (exact): every amplitude vs the dense vector."""
    circ, p = W.config_c1(seed)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=p["chi_max"])
    eps = m.run(circ)
    psi = dense.run_circuit(circ)
    amps = m.amplitudes(_all_bits(10))
    assert np.linalg.norm(amps - psi) / np.linalg.norm(psi) < 1e-10
    ref, recs = om.run_circuit(circ, p["chi_max"])
    assert list(m.bond_dims()) == ref.bond_dims()
    assert _spectrum_err(m, ref, 32) < 1e-10
    assert max(float(np.max(e)) for e in eps if len(e)) < 1e-20
    m.close()


def test_c1_complex64(T):
    circ, p = W.config_c1(1)
    m = T.MPS(10, dtype=T.TNSIM_C64, chi_max=p["chi_max"])
    m.run(circ)
    ref, _ = om.run_circuit(circ, p["chi_max"])
    assert 1 - _fidelity(m.export_sites(), ref.sites) <= 1e-6
    assert _spectrum_err(m, ref, 32) <= 1e-5
    m.close()


# ----------------------------------------------------------------- edge cases


@pytest.mark.parametrize("n,chi,cutoff,depth", [
    (2, 1, 0.0, 3), (2, 2, 0.0, 3), (3, 2, 0.0, 4), (5, 3, 0.0, 6), (12, 17, 0.0, 10),
    (13, 33, 0.0, 12), (9, 64, 1e-3, 8), (11, 5, 1e-2, 7),
])
def test_edge_shapes_complex128(T, n, chi, cutoff, depth):
    """Ragged and degenerate shapes: chi_max 1 (product state), odd widths, caps that are
    not powers of two, a binding cutoff."""
    circ = W.brickwork_u2_su4(n, depth, seed=n * 31 + chi)
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=chi, cutoff=cutoff)
    eps = m.run(circ)
    ref, recs = om.run_circuit(circ, chi, cutoff)
    assert list(m.bond_dims()) == ref.bond_dims()
    e_ref = np.array([r.eps for rr in recs for r in rr])
    e_got = np.concatenate([e for e in eps if len(e)])
    assert np.allclose(e_got, e_ref, rtol=1e-9, atol=1e-13)
    assert _spectrum_err(m, ref, chi) < 1e-10
    bits = W.random_bitstrings(n, 64, seed=n)
    a_ref = om.amplitudes(ref, bits)
    a_got = m.amplitudes(bits)
    assert np.linalg.norm(a_got - a_ref) <= 1e-10 * max(np.linalg.norm(a_ref), 1e-300)
    m.close()


def test_empty_and_one_qubit_only_layers(T):
    n = 7
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=8)
    ref = om.zero_state(n)
    rng = np.random.default_rng(5)
    u1 = np.stack([W.haar_unitary(2, rng) for _ in range(n)])
    lay0 = W.Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4)), u1)
    lay1 = W.Layer(np.array([1, 4], np.int32), np.stack([W.haar_su4(rng) for _ in range(2)]), u1)
    lay2 = W.Layer(np.zeros(0, np.int32), np.zeros((0, 4, 4)), None)
    for lay in (lay0, lay1, lay2, lay0):
        before = list(m.bond_dims())
        m.apply_layer(lay)
        om.apply_layer(ref, lay, 8)
        if lay.n2 == 0:
            assert list(m.bond_dims()) == before
    a = m.amplitudes(_all_bits(n))
    assert np.linalg.norm(a - om.to_dense(ref)) < 1e-12
    m.close()


def test_identity_gate_keeps_state(T):
    circ, p = W.config_c1(2)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=32)
    m.run(circ)
    before = m.amplitudes(_all_bits(10))
    eye = np.stack([np.eye(4, dtype=complex)] * 5)
    m.apply_layer(W.Layer(np.arange(0, 10, 2, dtype=np.int32), eye))
    after = m.amplitudes(_all_bits(10))
    assert np.linalg.norm(after - before) < 1e-12
    m.close()


def test_gate_set_with_fused_one_qubit_gates(T):
    """{H, CX, RZZ, RX} layers: one-qubit gates on paired qubits are fused into the 4x4
    on the device, the others update their site; checked against the dense vector."""
    circ = W.gateset_circuit(12, 14, seed=3)
    m = T.MPS(12, dtype=T.TNSIM_C128, chi_max=64)
    m.run(circ)
    psi = dense.run_circuit(circ)
    a = m.amplitudes(_all_bits(12))
    assert np.linalg.norm(a - psi) / np.linalg.norm(psi) < 1e-10
    m.close()


def test_ghz_and_qft_closed_forms(T):
    for n in (3, 8, 12):
        m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=16)
        m.run(W.ghz_circuit(n))
        a = m.amplitudes(np.array([[0] * n, [1] * n, [1] + [0] * (n - 1)], dtype=np.uint8))
        assert np.allclose(a, [2 ** -0.5, 2 ** -0.5, 0], atol=1e-14)
        assert max(m.bond_dims()) == 2
        m.close()
    n = 6
    x = [1, 0, 1, 1, 0, 1]
    m = T.MPS(n, dtype=T.TNSIM_C128, chi_max=64)
    m.run(W.qft_nn_circuit(n, x))
    a = m.amplitudes(_all_bits(n))
    assert np.allclose(np.abs(a), 2 ** (-n / 2), atol=1e-13)
    assert max(m.bond_dims()) == 1
    m.close()


# ----------------------------------------------------------------- schedules and variants


def test_plain_schedule_matches_batched_bitwise(T):
    circ = W.brickwork_su4(16, 10, seed=9)
    out = []
    for sched in (T.TNSIM_SCHED_BATCHED, T.TNSIM_SCHED_PLAIN):
        m = T.MPS(16, dtype=T.TNSIM_C64, chi_max=32, schedule=sched)
        m.run(circ)
        out.append(m.export_sites())
        m.close()
    for a, b in zip(*out):
        assert a.shape == b.shape and np.array_equal(a, b)


def test_device_gate_variant_matches_host_variant(T):
    torch = pytest.importorskip("torch")
    circ = W.brickwork_u2_su4(14, 8, seed=4)
    m1 = T.MPS(14, dtype=T.TNSIM_C64, chi_max=16)
    m1.run(circ)
    s = torch.cuda.Stream()
    m2 = T.MPS(14, dtype=T.TNSIM_C64, chi_max=16, stream=s.cuda_stream)
    eps_dev = torch.zeros(7, dtype=torch.float64, device="cuda")
    for lay in circ.layers:
        g = torch.from_numpy(np.ascontiguousarray(lay.g4).view(np.float64).copy()).cuda()
        u = torch.from_numpy(np.ascontiguousarray(lay.u1).view(np.float64).copy()).cuda()
        torch.cuda.synchronize()
        T.tnsim_apply_layer_device(m2.h, lay.pairs, g.data_ptr(), u.data_ptr(), eps_dev.data_ptr())
        m2.sync()
    for a, b in zip(m1.export_sites(), m2.export_sites()):
        assert np.array_equal(a, b)
    m1.close(); m2.close()


@pytest.mark.parametrize("mode", ["FP32", "FP32_3M", "TF32X3", "BF16X3"])
def test_contraction_modes_every_layer(T, mode):
    """Each complex64 contraction mode (FP32 4M / 3M on the FP32 pipe, 3xTF32 and BF16x3
    on tcgen05 tensor cores) against the oracle applied to the same input state, every
    layer of a 24-qubit chi 64 brickwork: singular values within 1e-5 of s_max, 1 - F <= 1e-6."""
    gm = getattr(T, "TNSIM_GEMM_" + mode)
    circ = W.brickwork_u2_su4(24, 10, seed=5)
    m = T.MPS(24, dtype=T.TNSIM_C64, chi_max=64, gemm=gm)
    for lay in circ.layers:
        pre = om.MPS(m.export_sites())
        m.apply_layer(lay)
        for r in om.apply_layer(pre, lay, 64):
            sg = m.spectrum(r.q + 1)
            k = max(len(sg), r.k)
            a = np.zeros(k); a[: len(sg)] = sg
            b = np.zeros(k); b[: r.k] = r.s_kept
            assert np.max(np.abs(a - b)) / r.s_kept[0] <= 1e-5
        assert 1 - om.fidelity(om.MPS(m.export_sites()), pre) <= 1e-6
    m.close()


@pytest.mark.parametrize("dt,tol", [("C128", 1e-10), ("C64", 1e-5)])
def test_plans_replayed_as_cuda_graphs(T, dt, tol):
    """Frozen layers (tnsim_plan) captured into CUDA graphs give the layer-by-layer
    result: (a) one graph of every layer, replayed once; (b) a graph of two layers
    (the even and the odd brickwork pattern) replayed four times with the gate buffers
    refreshed in between."""
    torch = pytest.importorskip("torch")
    dtype = getattr(T, "TNSIM_" + dt)
    circ = W.brickwork_u2_su4(14, 8, seed=12)
    ref = T.MPS(14, dtype=dtype, chi_max=16)
    ref.run(circ)
    want = ref.export_sites()
    stream = torch.cuda.Stream()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()

    # (a) all eight layers in one graph
    m = T.MPS(14, dtype=dtype, chi_max=16, stream=stream.cuda_stream)
    bufs = [(dev(l.g4), dev(l.u1)) for l in circ.layers]
    torch.cuda.synchronize()
    plans = [T.tnsim_plan_create([m.h], [(l.pairs, g.data_ptr(), u.data_ptr())])
             for l, (g, u) in zip(circ.layers, bufs)]
    graph = T.tnsim_graph_create(plans)
    T.tnsim_graph_launch(graph)
    m.sync()
    for a, b in zip(m.export_sites(), want):
        assert a.shape == b.shape
    assert 1 - _fidelity(m.export_sites(), want) <= (1e-12 if dt == "C128" else 1e-6)
    assert _spectrum_err(m, _spec_holder(ref), 16) <= tol
    T.tnsim_graph_destroy(graph)
    for p in plans:
        T.tnsim_plan_destroy(p)
    m.close()

    # (b) two layers, replayed with refreshed gates
    m = T.MPS(14, dtype=dtype, chi_max=16, stream=stream.cuda_stream)
    g_even, u_even = dev(circ.layers[0].g4), dev(circ.layers[0].u1)
    g_odd, u_odd = dev(circ.layers[1].g4), dev(circ.layers[1].u1)
    torch.cuda.synchronize()
    p_even = T.tnsim_plan_create([m.h], [(circ.layers[0].pairs, g_even.data_ptr(), u_even.data_ptr())])
    p_odd = T.tnsim_plan_create([m.h], [(circ.layers[1].pairs, g_odd.data_ptr(), u_odd.data_ptr())])
    graph = T.tnsim_graph_create([p_even, p_odd])
    for t in range(0, 8, 2):
        with torch.cuda.stream(stream):
            g_even.copy_(dev(circ.layers[t].g4)); u_even.copy_(dev(circ.layers[t].u1))
            g_odd.copy_(dev(circ.layers[t + 1].g4)); u_odd.copy_(dev(circ.layers[t + 1].u1))
        T.tnsim_graph_launch(graph)
    m.sync()
    assert 1 - _fidelity(m.export_sites(), want) <= (1e-12 if dt == "C128" else 1e-6)
    T.tnsim_graph_destroy(graph)
    T.tnsim_plan_destroy(p_even)
    T.tnsim_plan_destroy(p_odd)
    m.close()
    ref.close()


class _spec_holder:
    """Adapter: exposes a GPU state's bond spectra through the oracle MPS interface."""

    def __init__(self, m):
        self.n = m.n
        self.spectrum = [None] + [m.spectrum(b) if len(m.spectrum(b)) else None for b in range(1, m.n)] + [None]


# ----------------------------------------------------------------- failures stay on the host


def test_invalid_layers_are_rejected_without_touching_the_state(T):
    circ, _ = W.config_c1(3)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=32)
    m.run(circ)
    before = m.export_sites()
    g = np.stack([W.haar_su4(np.random.default_rng(0))] * 2)
    for q in ([0, 1], [8, 9], [-1, 3], [4, 4]):
        with pytest.raises(T.TnsimError) as ei:
            T.tnsim_apply_layer(m.h, np.array(q, np.int32), g)
        assert ei.value.status == T.TNSIM_EINVAL
    bad = g.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(T.TnsimError):
        T.tnsim_apply_layer(m.h, np.array([0, 4], np.int32), bad)
    for a, b in zip(before, m.export_sites()):
        assert np.array_equal(a, b)
    m.close()


def test_sweep_cap_reports_enoconv_and_keeps_going(T):
    circ = W.brickwork_su4(12, 8, seed=2)
    m = T.MPS(12, dtype=T.TNSIM_C64, chi_max=32, max_sweeps=1)
    with pytest.warns(T.TnsimConvergenceWarning):
        m.run(circ)
    m2 = T.MPS(12, dtype=T.TNSIM_C64, chi_max=32)   # the context is still usable
    m2.run(circ)
    ref, _ = om.run_circuit(circ, 32)
    assert 1 - _fidelity(m2.export_sites(), ref.sites) <= 1e-6
    m.close(); m2.close()


# ----------------------------------------------------------------- many states in one launch


def _steps_of(circs):
    depth = max(len(c.layers) for c in circs)
    steps = []
    for t in range(depth):
        row = []
        for c in circs:
            if t < len(c.layers):
                l = c.layers[t]
                row.append((l.pairs, l.g4, l.u1))
            else:
                row.append(None)
        steps.append(row)
    return steps


def test_batched_states_match_oracle_complex128(T):
    """Six circuits of uneven width, depth and chi_max, every step of every circuit in
    the same launches, against the oracle run circuit by circuit."""
    spec = [(8, 4, 4, 1), (12, 7, 8, 2), (16, 10, 16, 3), (20, 6, 32, 4), (10, 9, 8, 5), (14, 8, 16, 6)]
    circs = [W.brickwork_u2_su4(n, d, seed=s) for n, d, _, s in spec]
    ms = [T.MPS(n, dtype=T.TNSIM_C128, chi_max=chi) for n, _, chi, _ in spec]
    T.tnsim_apply_layers_batched([m.h for m in ms], _steps_of(circs))
    for (n, d, chi, _), c, m in zip(spec, circs, ms):
        ref, _ = om.run_circuit(c, chi)
        assert list(m.bond_dims()) == ref.bond_dims()
        assert _spectrum_err(m, ref, chi) < 1e-10
        bits = W.random_bitstrings(n, 64, seed=n)
        a_ref = om.amplitudes(ref, bits)
        assert np.linalg.norm(m.amplitudes(bits) - a_ref) <= 1e-10 * np.linalg.norm(a_ref)
        m.close()


@pytest.mark.slow
def test_c4_graph_captured_autotuned_batch(T):
    """The batching workload: 256 independent Haar SU(4) brickwork circuits (width
    U{16..128}, depth U{8..32}, chi_max in {16, 32, 64, 128, 256}, complex64, 3xTF32
    contraction).  Every step of every circuit is a frozen plan (all states' gates of
    that step in the same launches, one persistent Jacobi launch), the plans are
    captured into CUDA graphs and replayed; the Jacobi configuration is chosen by the
    autotuner on the largest state before the later plans are frozen.  At three
    steps a sample of 16 circuits spanning every chi_max bucket is checked against the
    oracle applied to its exported pre-step state (singular values within 1e-5 of
    s_max, discarded weights within 1e-5, 1 - F <= 1e-6), and the whole batch ends
    with every bond dimension inside its cap."""
    torch = pytest.importorskip("torch")
    batch = W.batch_circuits(256, base_seed=1000)
    circs = [c for c, _ in batch]
    chis = [chi for _, chi in batch]
    depth = max(len(c.layers) for c in circs)
    stream = torch.cuda.Stream()
    ms = [T.MPS(c.n_qubits, dtype=T.TNSIM_C64, chi_max=chi, gemm=T.TNSIM_GEMM_TF32X3, stream=stream.cuda_stream)
          for c, chi in batch]
    # every gate of every step on the device, once
    gdev = {}
    for i, c in enumerate(circs):
        for t, lay in enumerate(c.layers):
            gdev[(i, t)] = torch.from_numpy(np.ascontiguousarray(lay.g4).view(np.float64).copy()).cuda()
    torch.cuda.synchronize()

    def plan(t):
        idx = [i for i, c in enumerate(circs) if t < len(c.layers)]
        return T.tnsim_plan_create([ms[i].h for i in idx],
                                   [(circs[i].layers[t].pairs, gdev[(i, t)].data_ptr(), 0) for i in idx])

    def run_graph(steps):
        plans = [plan(t) for t in steps]
        if not plans:
            return
        g = T.tnsim_graph_create(plans)
        T.tnsim_graph_launch(g)
        ms[0].sync()
        T.tnsim_graph_destroy(g)
        for p in plans:
            T.tnsim_plan_destroy(p)

    checked = [5, 12, 20]
    deep = [i for i, c in enumerate(circs) if len(c.layers) > checked[-1]]
    sample = []
    for chi in (16, 32, 64, 128, 256):
        cand = sorted((i for i in deep if chis[i] == chi), key=lambda i: circs[i].n_qubits)
        sample += cand[:3]
    sample = sample[:16]
    assert len(sample) >= 15 and {chis[i] for i in sample} == {16, 32, 64, 128, 256}

    t0 = 0
    for tc in checked:
        run_graph(range(t0, tc))
        if tc == checked[0]:
            # autotune on the largest state's next layer, then freeze the remaining plans
            big = max(deep, key=lambda i: (chis[i], circs[i].n_qubits))
            lay = circs[big].layers[tc]
            choice, _ = T.tnsim_autotune(ms[big].h, lay.pairs, lay.g4, reps=1)
            for m in ms:
                T.tnsim_set_jacobi_config(m.h, choice)
        before = {i: ms[i].export_sites() for i in sample}
        run_graph([tc])
        for i in sample:
            ref = om.MPS(before[i])
            recs = om.apply_layer(ref, circs[i].layers[tc], chis[i])
            for r in recs:
                sg = ms[i].spectrum(r.q + 1)
                k = max(len(sg), r.k)
                a = np.zeros(k); a[: len(sg)] = sg
                b = np.zeros(k); b[: r.k] = r.s_kept
                assert np.max(np.abs(a - b)) / r.s_kept[0] <= 1e-5, (i, tc, r.q)
            assert 1 - om.fidelity(om.MPS(ms[i].export_sites()), ref) <= 1e-6, (i, tc)
        t0 = tc + 1
    run_graph(range(t0, depth))
    for i, (c, chi) in enumerate(batch):
        n = c.n_qubits
        cap = [min(chi, 2 ** min(b, n - b)) for b in range(n + 1)]
        got = list(ms[i].bond_dims())
        assert got[0] == got[n] == 1 and all(1 <= g_ <= w_ for g_, w_ in zip(got, cap)), i
    for m in ms:
        m.close()


# ----------------------------------------------------------------- read-out


def test_expect_pauli_matches_oracle(T):
    circ, p = W.config_c1(4)
    m = T.MPS(10, dtype=T.TNSIM_C128, chi_max=32)
    m.run(circ)
    ref, _ = om.run_circuit(circ, 32)
    rng = np.random.default_rng(8)
    terms = ["".join(rng.choice(list("IXYZ"), size=10)) for _ in range(10)]
    terms += ["I" * 10, "Z" + "I" * 9, "I" * 9 + "X"]
    terms += ["I" * i + "ZZ" + "I" * (8 - i) for i in range(9)]
    got = m.expect_pauli(terms)
    want = np.array([om.expect_pauli(ref, t) for t in terms])
    assert np.max(np.abs(got - want)) < 1e-10
    m.close()


# ----------------------------------------------------------------- the 64-qubit chi 128 workload
#
# Over many truncated layers any rounding is amplified: each truncation at chi_max
# projects onto the leading singular vectors, and with relative gaps at the cut of
# ~1e-3 a perturbation of theta tilts the kept subspace by ~1e3 times its size; once
# chi_max binds (layer 10) 1 - F grows ~3x per layer.  Even the precision floor of
# complex64 -- sites stored and contracted in complex64 around an exact FP64 SVD
# (oracle.mps.apply_2q_single_precision) -- reaches 1 - F = 1.5e-6 at layer 20.  So
# the complex64 tolerance is checked (a) per layer, for every layer, against the
# oracle applied to the GPU's own input state, and (b) end to end: at the stated
# tolerance through layer 16, and within a fixed factor of the precision floor
# after it.  The complex128 path is checked end to end over the whole depth.


def _c2_bits(ref):
    return np.concatenate([om.perfect_sample(ref, 1024, np.random.default_rng(1)),
                           W.random_bitstrings(ref.n, 64, seed=2)])


@pytest.mark.slow
def test_c2_complex128_end_to_end(T):
    """64 qubits, depth 20 Haar SU(4) brickwork, chi_max 128, cutoff 1e-10, complex128:
    per-bond singular values, 1024 sampled + 64 uniform amplitudes, <Z_i Z_i+1>, F."""
    circ, p = W.config_c2(1)
    m = T.MPS(64, dtype=T.TNSIM_C128, chi_max=p["chi_max"], cutoff=p["cutoff"])
    m.run(circ)
    ref, _ = om.run_circuit(circ, p["chi_max"], p["cutoff"])
    assert list(m.bond_dims()) == ref.bond_dims()
    assert _spectrum_err(m, ref, 128) <= 1e-10
    assert 1 - _fidelity(m.export_sites(), ref.sites) <= 1e-10
    bits = _c2_bits(ref)
    a_ref = om.amplitudes(ref, bits)
    assert np.linalg.norm(m.amplitudes(bits) - a_ref) / np.linalg.norm(a_ref) <= 1e-10
    zz = ["I" * i + "ZZ" + "I" * (62 - i) for i in range(63)]
    want = np.array([om.expect_pauli(ref, t) for t in zz])
    assert np.max(np.abs(m.expect_pauli(zz) - want)) <= 1e-10 * abs(om.norm2(ref))
    m.close()


@pytest.mark.slow
def test_c2_complex64_every_layer(T):
    """The same workload in complex64: every layer against the oracle applied to the
    GPU's own pre-layer state (singular values within 1e-5 of s_max, discarded
    weights, 1 - F <= 1e-6, amplitudes and <Z_i Z_i+1> of the last layer), and end
    to end against the oracle over the first 8 layers (the bonds reach 128 at layer 7)."""
    circ, p = W.config_c2(1)
    chi, cut = p["chi_max"], p["cutoff"]
    m = T.MPS(64, dtype=T.TNSIM_C64, chi_max=chi, cutoff=cut)
    ref = om.zero_state(64)
    for t, lay in enumerate(circ.layers):
        pre = om.MPS(m.export_sites())
        eps = m.apply_layer(lay)
        recs = om.apply_layer(pre, lay, chi, cut)
        for i, r in enumerate(recs):
            sg = m.spectrum(r.q + 1)
            k = max(len(sg), r.k)
            a = np.zeros(k); a[: len(sg)] = sg
            c = np.zeros(k); c[: r.k] = r.s_kept
            assert np.max(np.abs(a - c)) / r.s_kept[0] <= 1e-5, (t, r.q)
            assert abs(eps[i] - r.eps) <= 1e-5
        got = om.MPS(m.export_sites())
        assert 1 - om.fidelity(got, pre) <= 1e-6, t
        if t < 8:
            om.apply_layer(ref, lay, chi, cut)
            assert _spectrum_err(m, ref, chi) <= 1e-5
            assert 1 - om.fidelity(got, ref) <= 1e-6
    bits = _c2_bits(pre)
    a_ref = om.amplitudes(pre, bits)
    # |a - a_ref| / |a_ref| <= 2 sqrt(1 - F) with 1 - F <= 1e-6
    assert np.linalg.norm(m.amplitudes(bits) - a_ref) / np.linalg.norm(a_ref) <= 2e-3
    zz = ["I" * i + "ZZ" + "I" * (62 - i) for i in range(63)]
    n_ref, n_got = om.norm2(pre), om.norm2(got)
    want = np.array([om.expect_pauli(pre, t).real for t in zz]) / n_ref
    assert np.max(np.abs(m.expect_pauli(zz).real / n_got - want)) <= 2e-3
    m.close()


@pytest.mark.slow
def test_c2_complex64_end_to_end(T):
    """64 qubits, depth 20 Haar SU(4) brickwork, chi_max 128, cutoff 1e-10, complex64
    (default contraction and Jacobi tolerance) against the FP64 oracle run from
    |0...0>, layer after layer, next to the precision floor of complex64 (the
    oracle's single-precision variant, also against the FP64 oracle; at layer 20 the
    floor itself is at 1 - F = 6e-7 and 3e-5 of s_max on the singular values).
    Stated tolerance where the floor leaves room for it: 1 - F <= 1e-6 through layer
    16, singular values within 1e-5 of s_max through layer 12, and after layer 16 the
    1024 sampled + 64 uniform amplitudes and <Z_i Z_i+1> within 2e-3.  Later layers:
    1 - F within 150x and singular values within 30x the floor's."""
    circ, p = W.config_c2(1)
    chi, cut = p["chi_max"], p["cutoff"]
    m = T.MPS(64, dtype=T.TNSIM_C64, chi_max=chi, cutoff=cut)
    ref = om.zero_state(64)
    flo = om.zero_state(64)
    for t, lay in enumerate(circ.layers):
        m.apply_layer(lay)
        om.apply_layer(ref, lay, chi, cut)
        om.apply_layer(flo, lay, chi, cut, single=True)
        got = om.MPS(m.export_sites())
        inf = 1 - om.fidelity(got, ref)
        floor = 1 - om.fidelity(flo, ref)
        sp = _spectrum_err(m, ref, chi)
        sp_floor = _spectrum_err(_spec_holder_oracle(flo), ref, chi)
        if t < 12:
            assert sp <= 1e-5, (t, sp)
        else:
            assert sp <= max(1e-5, 30 * sp_floor), (t, sp, sp_floor)
        if t < 16:
            assert inf <= 1e-6, (t, inf)
        else:
            assert inf <= max(1e-6, 150 * floor), (t, inf, floor)
        if t == 15:
            bits = _c2_bits(ref)
            a_ref = om.amplitudes(ref, bits)
            assert np.linalg.norm(m.amplitudes(bits) - a_ref) / np.linalg.norm(a_ref) <= 2e-3
            zz = ["I" * i + "ZZ" + "I" * (62 - i) for i in range(63)]
            want = np.array([om.expect_pauli(ref, z).real for z in zz]) / om.norm2(ref)
            assert np.max(np.abs(m.expect_pauli(zz).real / om.norm2(got) - want)) <= 2e-3
    m.close()


class _spec_holder_oracle:
    """Adapter: exposes an oracle state's bond spectra through the GPU state's
    spectrum(bond) interface."""

    def __init__(self, mps):
        self.mps = mps

    def spectrum(self, b):
        s_ = self.mps.spectrum[b]
        return np.zeros(0) if s_ is None else s_


# ----------------------------------------------------------------- the gate-set workload (C3)


@pytest.mark.parametrize("mode", ["FP32_3M", "TF32X3", "BF16X3"])
def test_c3_gate_set_exact_width(T, mode):
    """{H, CX, RZZ(t), RX(t)} drawn per site, depth 24, chi_max 256, at 16 qubits where no
    bond can exceed 256: every contraction mode against the dense state vector."""
    circ = W.gateset_circuit(16, 24, seed=1)
    m = T.MPS(16, dtype=T.TNSIM_C64, chi_max=256, gemm=getattr(T, "TNSIM_GEMM_" + mode))
    m.run(circ)
    psi = dense.run_circuit(circ)
    got = om.to_dense(om.MPS(m.export_sites()))
    F = abs(np.vdot(got, psi)) ** 2 / (np.vdot(got, got).real * np.vdot(psi, psi).real)
    assert 1 - F <= 1e-6
    bits = W.random_bitstrings(16, 256, seed=4)
    idx = bits.astype(np.int64) @ (1 << np.arange(15, -1, -1))
    a = m.amplitudes(bits)
    assert np.linalg.norm(a - psi[idx]) / np.linalg.norm(psi[idx]) <= 2e-3
    m.close()


@pytest.mark.slow
def test_c3_full_size_last_layer(T):
    """100 qubits, depth 24, the gate set, chi_max 256, 3xTF32 contraction: the last layer
    (one-qubit draws fused or applied on their own, CX and RZZ pairs) against the oracle
    applied to the same exported input state -- every gate's kept singular values and the
    fidelity of the whole state after the layer."""
    circ, p = W.config_c3(1)
    m = T.MPS(100, dtype=T.TNSIM_C64, chi_max=p["chi_max"], gemm=T.TNSIM_GEMM_TF32X3)
    for lay in circ.layers[:-1]:
        m.apply_layer(lay)
    pre = om.MPS(m.export_sites())
    last = circ.layers[-1]
    m.apply_layer(last)
    recs = om.apply_layer(pre, last, p["chi_max"])
    for r in recs:
        sg = m.spectrum(r.q + 1)
        k = max(len(sg), r.k)
        a = np.zeros(k); a[: len(sg)] = sg
        b = np.zeros(k); b[: r.k] = r.s_kept
        assert np.max(np.abs(a - b)) / r.s_kept[0] <= 1e-5
    assert 1 - om.fidelity(om.MPS(m.export_sites()), pre) <= 1e-6
    m.close()


# ----------------------------------------------------------------- full size, sampled gates


@pytest.mark.slow
@pytest.mark.parametrize("cfg,gemm", [(0, "FP32"), (2, "TF32X3")])
def test_full_size_chi256_layer_sampled_gates(T, cfg, gemm):
    """100 qubits, chi_max 256, Haar SU(4) brickwork, complex64, in the batched launch
    of the benchmark (configuration 2 with the 3xTF32 contraction is what its
    autotuner picks; configuration 0 with FP32 is the default): after the bonds
    saturate, one more layer is applied on the GPU; for sampled pairs the oracle
    applies the same gate to the same (exported) input sites and the kept singular
    values, the discarded weight and the gauge-invariant two-site block
    A'_q A'_{q+1} are compared."""
    n, chi = 100, 256
    circ = W.brickwork_su4(n, 12, seed=7)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi, gemm=getattr(T, "TNSIM_GEMM_" + gemm))
    for lay in circ.layers[:11]:
        m.apply_layer(lay)
    assert int(np.max(m.bond_dims())) == chi
    T.tnsim_set_jacobi_config(m.h, cfg)
    before = m.export_sites()
    last = circ.layers[11]
    eps = m.apply_layer(last)
    after = m.export_sites()
    idx = [0, 3, len(last.pairs) // 2, len(last.pairs) - 1]
    for i in idx:
        q = int(last.pairs[i])
        mm = om.MPS([before[q], before[q + 1]])
        rec = om.apply_2q(mm, 0, last.g4[i], chi)
        s_gpu = m.spectrum(q + 1)
        assert len(s_gpu) == rec.k
        assert np.max(np.abs(s_gpu - rec.s_kept)) / rec.s_kept[0] <= 1e-5
        assert abs(eps[i] - rec.eps) <= 1e-5
        blk_ref = np.einsum("lxb,byr->lxyr", mm.sites[0], mm.sites[1])
        blk_gpu = np.einsum("lxb,byr->lxyr", after[q], after[q + 1])
        assert np.linalg.norm(blk_gpu - blk_ref) / np.linalg.norm(blk_ref) <= 1e-4
    m.close()


@pytest.fixture(scope="module")
def chi256_state(T):
    """A saturated 100-qubit chi 256 Haar brickwork state (11 layers, complex64) and
    the next layer."""
    n, chi = 100, 256
    circ = W.brickwork_su4(n, 12, seed=9)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi)
    for lay in circ.layers[:11]:
        m.apply_layer(lay)
    assert int(np.max(m.bond_dims())) == chi
    sites = m.export_sites()
    m.close()
    return sites, circ.layers[11]


@pytest.mark.slow
@pytest.mark.parametrize("mode,bound", [("FP32", 1e-6), ("FP32_3M", 5e-6), ("TF32X3", 1e-5), ("BF16X3", 1e-5)])
def test_c3_precision_modes_chi256(T, chi256_state, mode, bound):
    """The precision workload's per-result error at chi 256 (the gate-set circuit of C3
    never entangles beyond bond 16, so chi 256 comes from the Haar brickwork): every
    contraction arithmetic applies the same layer to the same saturated state, in the
    benchmark's launch configuration, and for 8 sampled gates the kept singular values
    are held to a per-mode bound (of s_max) against the oracle applied to the same
    input sites, the discarded weight to 1e-5, and the gauge-invariant two-site block
    to 1 - F <= 1e-6."""
    sites, lay = chi256_state
    n, chi = 100, 256
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi, gemm=getattr(T, "TNSIM_GEMM_" + mode))
    T.tnsim_set_jacobi_config(m.h, 2)
    m.import_sites(sites)
    eps = m.apply_layer(lay)
    after = m.export_sites()
    worst = 0.0
    for i in np.linspace(0, len(lay.pairs) - 1, 8).astype(int):
        q = int(lay.pairs[i])
        mm = om.MPS([sites[q], sites[q + 1]])
        rec = om.apply_2q(mm, 0, lay.g4[i], chi)
        s_gpu = m.spectrum(q + 1)
        assert len(s_gpu) == rec.k
        worst = max(worst, float(np.max(np.abs(s_gpu - rec.s_kept)) / rec.s_kept[0]))
        assert abs(eps[i] - rec.eps) <= 1e-5
        blk_ref = np.einsum("lxb,byr->lxyr", mm.sites[0], mm.sites[1])
        blk_gpu = np.einsum("lxb,byr->lxyr", after[q], after[q + 1])
        f = abs(np.vdot(blk_ref, blk_gpu)) ** 2 / (np.vdot(blk_ref, blk_ref).real * np.vdot(blk_gpu, blk_gpu).real)
        assert 1 - f <= 1e-6, (mode, q, 1 - f)
    assert worst <= bound, (mode, worst)
    m.close()
