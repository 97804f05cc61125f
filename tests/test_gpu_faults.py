"""Failure handling on the GPU: bounded waits that run out, and a device-memory cap.

No test here faults, traps or hangs the GPU.  A wait "runs out" because its poll
limit is set to a handful of polls (tnsim_set_wait_limits) while the event it waits
for still happens: the idle CTAs of the persistent Jacobi launch give up waiting
for a round of another CTA's gate, and the tensor-core contraction stops waiting
for TMA copies it issued, drains them with the default limit, and leaves.  Both
report status 5, which the synchronous call returns as ETIMEOUT.  Afterwards the
same handle (limits restored, sites imported) and a fresh handle run a correct
layer, which shows that the CUDA context stays usable.  ENOMEM comes from the
process-wide cap on device memory, checked before any allocation.
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


def _saturated(T, n, chi, depth, gemm):
    circ = W.brickwork_su4(n, depth + 1, seed=5)
    m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi, gemm=gemm)
    for lay in circ.layers[:depth]:
        m.apply_layer(lay)
    return m, circ.layers[depth]


def _check_layer(T, m, sites, lay, chi):
    """import the pre-layer sites, apply the layer, compare with the oracle"""
    m.import_sites(sites)
    m.apply_layer(lay)
    ref = om.MPS(sites)
    om.apply_layer(ref, lay, chi)
    assert 1 - om.fidelity(om.MPS(m.export_sites()), ref) <= 1e-6


@pytest.mark.parametrize("which", ["jacobi", "mbarrier"])
def test_bounded_wait_runs_out_then_context_is_usable(T, which):
    if which == "jacobi":
        # a 512 x 512 gate (16 visits per round, ~30 us each) beside a one-block gate that
        # finishes within microseconds: the launch has one CTA per visit of a round, so
        # once the small gate is done at least one CTA stays idle through every round of
        # the large one, and with a limit of one poll it gives up at its second poll
        n, chi = 20, 256
        m = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi)
        rng = np.random.default_rng(3)
        d = [min(2 ** b, 2 ** (n - b), chi) for b in range(n + 1)]
        m.import_sites([(rng.standard_normal((d[q], 2, d[q + 1])) + 1j * rng.standard_normal((d[q], 2, d[q + 1])))
                        / np.sqrt(4 * d[q + 1]) for q in range(n)])
        g = np.stack([W.haar_su4(rng) for _ in range(2)])
        lay = W.Layer(np.array([1, 9], np.int32), g, None)
        T.tnsim_set_wait_limits(m.h, 1, 0)
    else:
        n, chi = 16, 64
        m, lay = _saturated(T, n, chi, 8, T.TNSIM_GEMM_TF32X3)
        assert list(m.bond_dims())[6] == chi
        T.tnsim_set_wait_limits(m.h, 0, 1)     # one poll of each mbarrier wait
    sites = m.export_sites()
    got = []
    for _ in range(5):
        m.import_sites(sites)
        try:
            m.apply_layer(lay)
            got.append(T.TNSIM_OK)
        except T.TnsimError as e:
            got.append(e.status)
            assert "incomplete" in str(e) or "no progress" in str(e) or "wait" in str(e)
    assert set(got) <= {T.TNSIM_OK, T.TNSIM_ETIMEOUT}
    assert T.TNSIM_ETIMEOUT in got, got
    # the same handle with the default limits, then a fresh handle
    T.tnsim_set_wait_limits(m.h, 0, 0)
    _check_layer(T, m, sites, lay, chi)
    m2 = T.MPS(n, dtype=T.TNSIM_C64, chi_max=chi, gemm=m.params.gemm)
    _check_layer(T, m2, sites, lay, chi)
    m.close()
    m2.close()


def test_wait_limits_reject_bad_values(T):
    m = T.MPS(4, dtype=T.TNSIM_C64, chi_max=4)
    for a, b in ((-1, 0), (0, -1), (1 << 33, 0), (0, 1 << 31)):
        with pytest.raises(T.TnsimError) as ei:
            T.tnsim_set_wait_limits(m.h, a, b)
        assert ei.value.status == T.TNSIM_EINVAL
    m.close()


def test_device_memory_cap_gives_enomem_and_allocates_nothing(T):
    held0 = T.tnsim_device_bytes_held()
    small = T.MPS(8, dtype=T.TNSIM_C64, chi_max=8)
    held1 = T.tnsim_device_bytes_held()
    assert held1 > held0
    try:
        T.tnsim_set_device_memory_cap(held1 + (1 << 20))
        with pytest.raises(T.TnsimError) as ei:
            T.MPS(100, dtype=T.TNSIM_C64, chi_max=256)          # ~0.3 GB
        assert ei.value.status == T.TNSIM_ENOMEM and "cap" in str(ei.value)
        assert T.tnsim_device_bytes_held() == held1
        ok = T.MPS(6, dtype=T.TNSIM_C64, chi_max=4)               # fits under the cap
        ok.close()
        assert T.tnsim_device_bytes_held() == held1
    finally:
        T.tnsim_set_device_memory_cap(0)
    big = T.MPS(100, dtype=T.TNSIM_C64, chi_max=256)
    big.run(W.brickwork_su4(100, 2, seed=1))
    big.close()
    small.close()
    assert T.tnsim_device_bytes_held() == held0
    with pytest.raises(T.TnsimError):
        T.tnsim_set_device_memory_cap(-1)
