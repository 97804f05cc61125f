"""Reverse-mode energy gradient on the GPU (tnsim_grad) against the oracle (oracle/grad.py).

The oracle's gradient is the exact derivative of the truncated simulation and is
itself pinned by finite differences (tests/test_grad_cpu.py).  Both sides use the
same pseudo-inverse cutoff tau = sqrt(eps) of the arithmetic (singular directions
below tau s_max get no inverse factors).  Tolerances: complex128 within 1e-9 of the
largest component (energy 1e-12); complex64 within 2e-3 (energy 1e-5 relative).
At a binding cut with degenerate singular values the truncated energy is not
differentiable (which of the degenerate vectors is kept depends on rounding); the
50-qubit workload runs with a 1e-10 discarded-weight cutoff that drops the
numerically zero directions (tests/hea_workload.py), and there every component is
compared, and the oracle is pinned by finite differences at that workload.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import grad as OG

pytestmark = pytest.mark.gpu

TAU64, TAU32 = float(np.finfo(np.float64).eps) ** 0.5, float(np.finfo(np.float32).eps) ** 0.5


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    return T


def _hea(n, n_layers, seed, sigma):
    circ, angles = W.hea_circuit(n, n_layers, seed=seed, sigma=sigma)
    layers = [(l.pairs, l.g4) for l in circ.layers]
    axes = ["YZ" if i % 2 == 0 else "" for i in range(len(layers))]
    theta = [angles[i // 2].copy() if i % 2 == 0 else np.zeros((n, 0)) for i in range(len(layers))]
    paulis = ["".join("Z" if k in (i, i + 1) else "I" for k in range(n)) for i in range(n - 1)] + \
             ["".join("X" if k == i else "I" for k in range(n)) for i in range(n)]
    coeffs = [1.0] * (n - 1) + [0.5] * n
    return layers, axes, theta, paulis, coeffs


def _params(T, dtype, chi, renorm=True):
    p = T.tnsim_params_default(dtype)
    p.chi_max, p.renormalize = chi, int(renorm)
    return p


def _flat(gs):
    return np.concatenate([g.reshape(-1) for g in gs])


@pytest.mark.parametrize("chi,renorm", [(64, True), (4, True), (3, True), (3, False)])
def test_complex128_against_the_oracle(T, chi, renorm):
    n = 8
    layers, axes, theta, paulis, coeffs = _hea(n, 4, seed=3, sigma=0.5)
    e, g = T.tnsim_grad(n, layers, axes, theta, paulis, coeffs, T.TNSIM_C128, _params(T, T.TNSIM_C128, chi, renorm))
    e_ref, g_ref = OG.grad(n, layers, axes, theta, paulis, coeffs, chi_max=chi, renormalize=renorm, tau=TAU64,
                           broaden=TAU64 ** 4)
    assert abs(e - e_ref) < 1e-12
    gf, rf = _flat(g), _flat(g_ref)
    assert np.max(np.abs(gf - rf)) <= 1e-9 * np.max(np.abs(rf))


def test_complex128_against_finite_differences_of_its_own_energy(T):
    n, chi = 8, 3
    layers, axes, theta, paulis, coeffs = _hea(n, 3, seed=5, sigma=0.6)
    p = _params(T, T.TNSIM_C128, chi)
    e, g = T.tnsim_grad(n, layers, axes, theta, paulis, coeffs, T.TNSIM_C128, p)
    h = 1e-6
    for L, q, j in [(0, 0, 0), (0, 3, 1), (2, 5, 0), (4, 7, 1), (4, 2, 0)]:
        tp = [t.copy() for t in theta]; tm = [t.copy() for t in theta]
        tp[L][q, j] += h; tm[L][q, j] -= h
        ep, _ = T.tnsim_grad(n, layers, axes, tp, paulis, coeffs, T.TNSIM_C128, p)
        em, _ = T.tnsim_grad(n, layers, axes, tm, paulis, coeffs, T.TNSIM_C128, p)
        assert abs((ep - em) / (2 * h) - g[L][q, j]) < 1e-7


@pytest.mark.parametrize("n,chi", [(10, 32), (12, 16)])
def test_complex64_against_the_oracle(T, n, chi):
    layers, axes, theta, paulis, coeffs = _hea(n, 4, seed=7, sigma=0.5)
    e, g = T.tnsim_grad(n, layers, axes, theta, paulis, coeffs, T.TNSIM_C64, _params(T, T.TNSIM_C64, chi))
    e_ref, g_ref = OG.grad(n, layers, axes, theta, paulis, coeffs, chi_max=chi, tau=TAU32, broaden=TAU32 ** 4)
    assert abs(e - e_ref) < 1e-5 * max(1.0, abs(e_ref))
    gf, rf = _flat(g), _flat(g_ref)
    assert np.max(np.abs(gf - rf)) <= 2e-3 * np.max(np.abs(rf))


@pytest.mark.slow
def test_hea_workload_gradient(T):
    """The differentiation workload (tests/hea_workload.py: 50 qubits, 10 HEA layers,
    1000 angles, chi_max 64, cutoff 1e-10, seed 2):
      1. the oracle's exact gradient against central finite differences (h = 1e-4,
         FP64) of its own energy on 32 seeded angles, within 1e-5 of the largest
         component (measured 3e-7);
      2. complex128 on the GPU: the energy within 1e-10 relative and every one of the
         1000 components within 1e-5 of the largest, against the oracle with the same
         regularisation (pseudo-inverse cutoff sqrt(eps) s_max, broadening eps^2);
         central differences of the GPU's own energy on 4 angles within 1e-6;
      3. complex64 on the GPU (oracle with the FP32 regularisation): the energy within
         1e-5 relative.  The gradient is compared component by component only with a
         cutoff of 1e-4, where every kept singular value is above ~1e-2 s_max: there
         every component lies within 1e-3 of the largest (measured 1.6e-4).  With the
         workload's cutoff of 1e-10 the kept directions reach down to ~1e-5 s_max,
         below what FP32 singular vectors resolve, and the adjoint of those directions
         (1 / s factors, couplings across the cut) is not reproducible in complex64:
         72 % of the components agree within 1e-3 of the largest, the worst by 0.4."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import hea_workload as H

    n = H.N
    layers, axes, theta, paulis, coeffs = H.hea()
    rng = np.random.default_rng(7)
    picks = [(2 * int(rng.integers(H.N_LAYERS)), int(rng.integers(n)), int(rng.integers(2))) for _ in range(32)]
    h = 1e-4
    args = [(L, q, j, s * h) for (L, q, j) in picks for s in (1.0, -1.0)]
    # one BLAS thread per worker process (the variables are read when a worker loads numpy)
    one = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    saved = {k: os.environ.get(k) for k in one}
    os.environ.update(one)
    try:
        with ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)),
                                 mp_context=mp.get_context("spawn")) as ex:
            es = list(ex.map(H.energy_shifted, args))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    fd = np.array([(es[2 * i] - es[2 * i + 1]) / (2 * h) for i in range(len(picks))])
    e_ex, g_ex = OG.grad(n, layers, axes, theta, paulis, coeffs, chi_max=H.CHI, cutoff=H.CUTOFF)
    gmax = np.max(np.abs(_flat(g_ex)))
    want = np.array([g_ex[L][q, j] for (L, q, j) in picks])
    assert np.max(np.abs(fd - want)) <= 1e-5 * gmax, np.max(np.abs(fd - want)) / gmax

    cases = ((T.TNSIM_C128, H.CUTOFF, TAU64, 1e-10, 1e-5),
             (T.TNSIM_C64, H.CUTOFF, TAU32, 1e-5, None),
             (T.TNSIM_C64, 1e-4, TAU32, 1e-5, 1e-3))
    for dt, cut, tau, tol_e, tol_g in cases:
        p = _params(T, dt, H.CHI)
        p.cutoff = cut
        e, g = T.tnsim_grad(n, layers, axes, theta, paulis, coeffs, dt, p)
        e_ref, g_ref = OG.grad(n, layers, axes, theta, paulis, coeffs, chi_max=H.CHI, cutoff=cut, tau=tau,
                               broaden=tau ** 4)
        gf, rf = _flat(g), _flat(g_ref)
        assert gf.size == 1000 and np.all(np.isfinite(gf))
        assert abs(e - e_ref) <= tol_e * abs(e_ref), (dt, e, e_ref)
        if tol_g is not None:
            err = np.max(np.abs(gf - rf)) / np.max(np.abs(rf))
            assert err <= tol_g, (dt, cut, err)
        if dt == T.TNSIM_C128:
            for (L, q, j) in picks[:4]:
                tp = [t.copy() for t in theta]; tm = [t.copy() for t in theta]
                tp[L][q, j] += h; tm[L][q, j] -= h
                ep, _ = T.tnsim_grad(n, layers, axes, tp, paulis, coeffs, dt, p)
                em, _ = T.tnsim_grad(n, layers, axes, tm, paulis, coeffs, dt, p)
                assert abs((ep - em) / (2 * h) - g[L][q, j]) <= 1e-6 * np.max(np.abs(rf))


def test_torch_autograd_function(T):
    torch = pytest.importorskip("torch")
    from paper_2601_04422_gb300.autograd import circuit_energy
    n = 6
    layers, axes, theta, paulis, coeffs = _hea(n, 2, seed=9, sigma=0.4)
    flat = torch.tensor(_flat(theta), dtype=torch.float64, requires_grad=True)
    e = circuit_energy(flat, n, layers, axes, paulis, coeffs, T.TNSIM_C128, _params(T, T.TNSIM_C128, 16))
    (3.0 * e).backward()
    e_ref, g_ref = OG.grad(n, layers, axes, theta, paulis, coeffs, chi_max=16)
    assert abs(e.item() - e_ref) < 1e-12
    assert np.max(np.abs(flat.grad.numpy() - 3.0 * _flat(g_ref))) < 1e-9


def test_bad_arguments(T):
    n = 4
    layers, axes, theta, paulis, coeffs = _hea(n, 1, seed=1, sigma=0.3)
    with pytest.raises(T.TnsimError) as ei:
        T.tnsim_grad(n, layers, axes, theta, ["ZZIA"], [1.0], T.TNSIM_C128)
    assert ei.value.status == T.TNSIM_EINVAL
    p = _params(T, T.TNSIM_C128, 8)
    p.form = T.TNSIM_FORM_CANONICAL
    with pytest.raises(T.TnsimError) as ei:
        T.tnsim_grad(n, layers, axes, theta, paulis, coeffs, T.TNSIM_C128, p)
    assert ei.value.status == T.TNSIM_EUNSUPPORTED
