"""ctypes marshalling for libtnsim.so: one Python function per C entry point, same names.

Host arrays are numpy arrays (complex gates are passed as complex128 and viewed as
interleaved doubles).  Device buffers are raw pointers (ints), e.g. from
``torch.Tensor.data_ptr()``; streams are ``cudaStream_t`` values as ints (e.g.
``torch.cuda.Stream.cuda_stream``) or None for a library-owned stream.
"""
from __future__ import annotations

import ctypes as C
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libtnsim.so")

TNSIM_OK, TNSIM_EINVAL, TNSIM_ENOMEM, TNSIM_ECUDA, TNSIM_ENOCONV, TNSIM_ETIMEOUT, TNSIM_EUNSUPPORTED = range(7)
TNSIM_C64, TNSIM_C128 = 0, 1
TNSIM_SCHED_BATCHED, TNSIM_SCHED_PLAIN = 0, 1
TNSIM_GEMM_FP32, TNSIM_GEMM_FP32_3M, TNSIM_GEMM_TF32X3, TNSIM_GEMM_BF16X3 = 0, 1, 2, 3
TNSIM_FORM_PAPER, TNSIM_FORM_CANONICAL = 0, 1

_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}


class TnsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tnsim {_NAMES.get(status, status)}: {msg}")
        self.status = status


class TnsimConvergenceWarning(RuntimeWarning):
    pass


if not os.path.exists(lib_path):
    raise ImportError(
        f"{lib_path} is missing: build it with __graft_entry__.build() or "
        "python paper_2601_04422_gb300/build.py (the library has no CPU fallback)")

lib = C.CDLL(lib_path)


class tnsim_params(C.Structure):
    _fields_ = [("chi_max", C.c_int32), ("cutoff", C.c_double), ("renormalize", C.c_int32),
                ("max_sweeps", C.c_int32), ("jacobi_tol", C.c_double), ("schedule", C.c_int32),
                ("gemm", C.c_int32), ("form", C.c_int32)]


_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_DP = C.POINTER(C.c_double)


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("tnsim_params_default", C.c_int, [C.c_int, C.POINTER(tnsim_params)])
_sig("tnsim_mps_create", C.c_int, [C.c_int32, C.c_int, C.POINTER(tnsim_params), _P, C.POINTER(_P)])
_sig("tnsim_mps_destroy", C.c_int, [_P])
_sig("tnsim_apply_layer", C.c_int, [_P, C.c_int32, _I32P, _DP, _DP, _DP])
_sig("tnsim_apply_layer_device", C.c_int, [_P, C.c_int32, _I32P, _P, _P, _P])
_sig("tnsim_apply_layers_batched", C.c_int,
     [C.POINTER(_P), C.c_int32, C.c_int32, _I32P, C.POINTER(_I32P), C.POINTER(_DP), C.POINTER(_DP)])
_sig("tnsim_sync", C.c_int, [_P])
_sig("tnsim_bond_dims", C.c_int, [_P, _I32P])
_sig("tnsim_bond_spectrum", C.c_int, [_P, C.c_int32, _DP, _I32P])
_sig("tnsim_export_sites", C.c_int, [_P, _DP, C.c_int64, _I64P])
_sig("tnsim_import_sites", C.c_int, [_P, _I32P, _DP])
_sig("tnsim_amplitudes", C.c_int, [_P, C.c_int64, C.POINTER(C.c_uint8), _DP])
_sig("tnsim_expect_pauli", C.c_int, [_P, C.c_int32, C.c_char_p, _DP])
class tnsim_circuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_layers", C.c_int32), ("n_rot", _I32P), ("axes", C.c_char_p),
                ("n2", _I32P), ("q", _I32P), ("g4x4", _DP)]


class tnsim_hamiltonian(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("paulis", C.c_char_p), ("coeffs", _DP)]


_sig("tnsim_grad", C.c_int, [C.POINTER(tnsim_circuit), _DP, C.POINTER(tnsim_hamiltonian), C.c_int,
                             C.POINTER(tnsim_params), _P, _DP, _DP])
class tnsim_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("gates", "sweeps", "rotations", "pair_visits", "visit_rows",
                                          "rotation_rows", "theta_cmacs", "right_cmacs", "qr_cmacs")]


TNSIM_K_NAMES = ["site1q", "theta", "jacobi", "truncate", "left", "right", "qr"]

_sig("tnsim_last_stats", C.c_int, [_P, C.POINTER(tnsim_stats)])
_sig("tnsim_profile_enable", C.c_int, [_P, C.c_int32])
_sig("tnsim_profile_read", C.c_int, [_P, _DP, _I64P])
_sig("tnsim_two_site_update_noalloc", C.c_int,
     [_P, C.c_int64, _P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _DP, C.c_int32, C.c_double,
      C.c_int32, _P, _I32P, _DP, _DP])
_sig("tnsim_plan_create", C.c_int, [C.POINTER(_P), C.c_int32, _I32P, C.POINTER(_I32P), C.POINTER(_P),
                                     C.POINTER(_P), C.POINTER(_P)])
_sig("tnsim_plan_launch", C.c_int, [_P])
_sig("tnsim_plan_destroy", C.c_int, [_P])
_sig("tnsim_graph_create", C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(_P)])
_sig("tnsim_graph_launch", C.c_int, [_P])
_sig("tnsim_graph_destroy", C.c_int, [_P])
_sig("tnsim_apply_circuit", C.c_int, [_P, C.c_int32, _I32P, _I32P, _DP, _I32P, _I32P, _DP])
_sig("tnsim_circuit_layerize", C.c_int, [C.c_int32, C.c_int32, _I32P, _I32P, _DP, C.c_int32, C.c_int32,
                                         _I32P, _I32P, _I32P, _I32P, _DP, _DP])
_sig("tnsim_sample", C.c_int, [_P, C.c_int64, _DP, C.POINTER(C.c_uint8), _I64P])
_sig("tnsim_set_jacobi_config", C.c_int, [_P, C.c_int32])
_sig("tnsim_set_wait_limits", C.c_int, [_P, C.c_int64, C.c_int64])
_sig("tnsim_set_device_memory_cap", C.c_int, [C.c_int64])
_sig("tnsim_device_bytes_held", C.c_int64, [])
_sig("tnsim_autotune", C.c_int, [_P, C.c_int32, _I32P, _DP, C.c_int32, _I32P, _DP])
_sig("tnsim_last_error", C.c_char_p, [])
_sig("tnsim_version", C.c_char_p, [])


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return ["tnsim_params_default", "tnsim_mps_create", "tnsim_mps_destroy", "tnsim_apply_layer",
            "tnsim_apply_layer_device", "tnsim_apply_layers_batched", "tnsim_sync",
            "tnsim_bond_dims", "tnsim_bond_spectrum", "tnsim_export_sites", "tnsim_import_sites",
            "tnsim_amplitudes", "tnsim_expect_pauli", "tnsim_grad", "tnsim_last_stats",
            "tnsim_profile_enable", "tnsim_profile_read", "tnsim_two_site_update_noalloc",
            "tnsim_plan_create", "tnsim_plan_launch", "tnsim_plan_destroy", "tnsim_graph_create",
            "tnsim_graph_launch", "tnsim_graph_destroy", "tnsim_apply_circuit", "tnsim_circuit_layerize", "tnsim_sample", "tnsim_set_jacobi_config",
            "tnsim_autotune", "tnsim_set_wait_limits", "tnsim_set_device_memory_cap", "tnsim_device_bytes_held",
            "tnsim_last_error", "tnsim_version"]


def tnsim_last_error() -> str:
    return lib.tnsim_last_error().decode()


def tnsim_version() -> str:
    return lib.tnsim_version().decode()


def _check(st: int):
    if st == TNSIM_OK:
        return
    msg = tnsim_last_error()
    if st == TNSIM_ENOCONV:
        warnings.warn(msg, TnsimConvergenceWarning, stacklevel=3)
        return
    raise TnsimError(st, msg)


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _cplx(a, shape_tail):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.reshape((-1,) + shape_tail)


def tnsim_params_default(dtype: int = TNSIM_C64) -> tnsim_params:
    p = tnsim_params()
    _check(lib.tnsim_params_default(dtype, C.byref(p)))
    return p


def tnsim_mps_create(n_qubits: int, dtype: int = TNSIM_C64, params: tnsim_params = None, stream=None):
    h = _P()
    _check(lib.tnsim_mps_create(int(n_qubits), int(dtype), C.byref(params) if params is not None else None,
                                _P(int(stream)) if stream else None, C.byref(h)))
    return h


def tnsim_mps_destroy(h):
    _check(lib.tnsim_mps_destroy(h))


def tnsim_apply_layer(h, q, g4x4, u1=None):
    """Apply one layer; returns the discarded weight of every gate (numpy float64)."""
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    n2 = q.shape[0]
    g = _cplx(g4x4, (4, 4)) if n2 else np.zeros((0, 4, 4), np.complex128)
    assert g.shape[0] == n2
    u = _cplx(u1, (2, 2)) if u1 is not None else None
    eps = np.zeros(max(n2, 1), dtype=np.float64)
    gd = g.view(np.float64)
    ud = u.view(np.float64) if u is not None else None
    _check(lib.tnsim_apply_layer(h, n2, q.ctypes.data_as(_I32P), _dptr(gd), _dptr(ud), _dptr(eps)))
    return eps[:n2]


def tnsim_apply_layer_device(h, q, g4x4_dev: int, u1_dev: int = 0, eps_dev: int = 0):
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    _check(lib.tnsim_apply_layer_device(h, q.shape[0], q.ctypes.data_as(_I32P), _P(g4x4_dev or None),
                                        _P(u1_dev or None), _P(eps_dev or None)))


def _ops_arrays(ops):
    """ops: sequence of (qa, qb, matrix) with qb None or < 0 for a one-qubit gate (2x2)."""
    n = len(ops)
    qa = np.zeros(max(n, 1), np.int32)
    qb = np.zeros(max(n, 1), np.int32)
    mats = np.zeros((max(n, 1), 16), np.complex128)
    for i, (a, b, g) in enumerate(ops):
        g = np.asarray(g, dtype=np.complex128)
        qa[i] = int(a)
        if b is None or int(b) < 0:
            qb[i] = -1
            mats[i, :4] = g.reshape(4)
        else:
            qb[i] = int(b)
            mats[i] = g.reshape(16)
    return n, qa, qb, mats.view(np.float64)


def tnsim_apply_circuit(h, ops):
    """Apply a gate list on any qubits; returns (n_layers, n_local_gates, eps_sum)."""
    n, qa, qb, md = _ops_arrays(ops)
    nl, ng, eps = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    _check(lib.tnsim_apply_circuit(h, n, qa.ctypes.data_as(_I32P), qb.ctypes.data_as(_I32P), _dptr(md),
                                   C.byref(nl), C.byref(ng), C.byref(eps)))
    return nl.value, ng.value, eps.value


def tnsim_circuit_layerize(n_qubits: int, ops):
    """The host planner alone: returns a list of layers (pairs, g4 [n2,4,4], u1 [n,2,2])."""
    n, qa, qb, md = _ops_arrays(ops)
    nl, ng = C.c_int32(0), C.c_int32(0)
    args = (int(n_qubits), n, qa.ctypes.data_as(_I32P), qb.ctypes.data_as(_I32P), _dptr(md))
    _check(lib.tnsim_circuit_layerize(*args, 0, 0, C.byref(nl), C.byref(ng), None, None, None, None))
    L, G = nl.value, ng.value
    n2 = np.zeros(max(L, 1), np.int32)
    gq = np.zeros(max(G, 1), np.int32)
    g4 = np.zeros((max(G, 1), 4, 4), np.complex128)
    u1 = np.zeros((max(L, 1), int(n_qubits), 2, 2), np.complex128)
    _check(lib.tnsim_circuit_layerize(*args, L, G, C.byref(nl), C.byref(ng), n2.ctypes.data_as(_I32P),
                                      gq.ctypes.data_as(_I32P), _dptr(g4.view(np.float64)),
                                      _dptr(u1.view(np.float64))))
    out, off = [], 0
    for i in range(L):
        k = int(n2[i])
        out.append((gq[off:off + k].copy(), g4[off:off + k].copy(), u1[i].copy()))
        off += k
    return out


def tnsim_apply_layers_batched(handles, steps):
    """steps[t][i] = (q, g4x4, u1) or None for state i at step t."""
    n_circ, n_steps = len(handles), len(steps)
    hs = (_P * n_circ)(*[h.value if isinstance(h, _P) else h for h in handles])
    tot = n_circ * n_steps
    n2 = np.zeros(tot, dtype=np.int32)
    qp = (_I32P * tot)()
    gp = (_DP * tot)()
    up = (_DP * tot)()
    keep = []
    for t, row in enumerate(steps):
        for i, item in enumerate(row):
            k = t * n_circ + i
            if item is None:
                continue
            q, g, u = item
            q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
            n2[k] = q.shape[0]
            gd = _cplx(g, (4, 4)).view(np.float64) if q.shape[0] else np.zeros(1)
            keep += [q, gd]
            qp[k] = q.ctypes.data_as(_I32P)
            gp[k] = gd.ctypes.data_as(_DP)
            if u is not None:
                ud = _cplx(u, (2, 2)).view(np.float64)
                keep.append(ud)
                up[k] = ud.ctypes.data_as(_DP)
    _check(lib.tnsim_apply_layers_batched(hs, n_circ, n_steps, n2.ctypes.data_as(_I32P), qp, gp, up))


def tnsim_sync(h):
    _check(lib.tnsim_sync(h))


def tnsim_bond_dims(h, n_qubits: int) -> np.ndarray:
    out = np.zeros(n_qubits + 1, dtype=np.int32)
    _check(lib.tnsim_bond_dims(h, out.ctypes.data_as(_I32P)))
    return out


def tnsim_bond_spectrum(h, bond: int, chi_max: int) -> np.ndarray:
    s = np.zeros(chi_max, dtype=np.float64)
    k = C.c_int32(0)
    _check(lib.tnsim_bond_spectrum(h, int(bond), _dptr(s), C.byref(k)))
    return s[: k.value].copy()


def tnsim_export_sites(h, n_qubits: int):
    """Returns the list of site tensors (complex128, shapes (chi_q, 2, chi_{q+1}))."""
    need = C.c_int64(0)
    _check(lib.tnsim_export_sites(h, None, 0, C.byref(need)))
    buf = np.zeros(need.value, dtype=np.float64)
    _check(lib.tnsim_export_sites(h, _dptr(buf), need.value, C.byref(need)))
    dims = tnsim_bond_dims(h, n_qubits)
    z = buf.view(np.complex128)
    sites, pos = [], 0
    for q in range(n_qubits):
        cnt = int(dims[q]) * 2 * int(dims[q + 1])
        sites.append(z[pos:pos + cnt].reshape(int(dims[q]), 2, int(dims[q + 1])).copy())
        pos += cnt
    return sites


def tnsim_import_sites(h, sites):
    dims = np.array([1] + [s.shape[2] for s in sites], dtype=np.int32)
    data = np.concatenate([np.ascontiguousarray(s, dtype=np.complex128).reshape(-1) for s in sites])
    dd = data.view(np.float64)
    _check(lib.tnsim_import_sites(h, dims.ctypes.data_as(_I32P), _dptr(dd)))


def tnsim_amplitudes(h, bits) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    n_str = bits.shape[0]
    out = np.zeros(2 * max(n_str, 1), dtype=np.float64)
    _check(lib.tnsim_amplitudes(h, n_str, bits.ctypes.data_as(C.POINTER(C.c_uint8)), _dptr(out)))
    return out[: 2 * n_str].view(np.complex128).copy()


def tnsim_expect_pauli(h, paulis) -> np.ndarray:
    terms = list(paulis)
    blob = "".join(terms).encode()
    out = np.zeros(2 * max(len(terms), 1), dtype=np.float64)
    _check(lib.tnsim_expect_pauli(h, len(terms), blob, _dptr(out)))
    return out[: 2 * len(terms)].view(np.complex128).copy()


def tnsim_sample(h, uniforms):
    """Perfect sampling with the given uniforms [n_shots, n_qubits] in [0, 1);
    returns (bits uint8 [n_shots, n_qubits], distinct prefixes evaluated)."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    assert u.ndim == 2
    bits = np.zeros(u.shape, dtype=np.uint8)
    nodes = C.c_int64(0)
    _check(lib.tnsim_sample(h, u.shape[0], _dptr(u), bits.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(nodes)))
    return bits, nodes.value


TNSIM_JACOBI_CONFIGS = 8


def tnsim_set_jacobi_config(h, cfg: int):
    _check(lib.tnsim_set_jacobi_config(h, int(cfg)))


def tnsim_set_wait_limits(h, jacobi_idle_polls: int = 0, mbarrier_polls: int = 0):
    """Poll limits of the bounded device waits (0 = defaults)."""
    _check(lib.tnsim_set_wait_limits(h, int(jacobi_idle_polls), int(mbarrier_polls)))


def tnsim_set_device_memory_cap(nbytes: int):
    """Process-wide cap on the device bytes held by states (0 = none)."""
    _check(lib.tnsim_set_device_memory_cap(int(nbytes)))


def tnsim_device_bytes_held() -> int:
    return int(lib.tnsim_device_bytes_held())


def tnsim_autotune(h, q, g4x4, reps: int = 3):
    """Time every Jacobi configuration on one layer; returns (choice, ms per configuration)."""
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
    g = _cplx(g4x4, (4, 4))
    choice = C.c_int32(0)
    ms = np.zeros(TNSIM_JACOBI_CONFIGS, dtype=np.float64)
    _check(lib.tnsim_autotune(h, q.shape[0], q.ctypes.data_as(_I32P), _dptr(g.view(np.float64)), int(reps),
                              C.byref(choice), _dptr(ms)))
    return choice.value, ms


def tnsim_grad(n_qubits: int, layers, axes, theta, paulis, coeffs, dtype: int = TNSIM_C128, params=None,
               stream=None):
    """Energy and angle gradient of a layered circuit (reverse mode through the simulation).

    layers[L] = (pairs, g4 [n2, 4, 4]); axes[L] a string of rotation axes (first acts
    first); theta[L] an array [n_qubits, len(axes[L])]; H = sum coeffs[t] * paulis[t].
    Returns (E, [dE/dtheta_L])."""
    n, nl = int(n_qubits), len(layers)
    n_rot = np.array([len(a) for a in axes] or [0], dtype=np.int32)
    n2 = np.array([len(np.asarray(pq).reshape(-1)) for pq, _ in layers] or [0], dtype=np.int32)
    q = np.concatenate([np.asarray(pq, dtype=np.int32).reshape(-1) for pq, _ in layers] + [np.zeros(1, np.int32)])
    g = np.concatenate([_cplx(g4, (4, 4)).reshape(-1, 4, 4) for _, g4 in layers if len(g4)] +
                       [np.zeros((1, 4, 4), np.complex128)])
    th = np.concatenate([np.asarray(t, dtype=np.float64).reshape(-1) for t in theta] + [np.zeros(1)])
    ax = "".join(axes).encode()
    c = tnsim_circuit(n, nl, n_rot.ctypes.data_as(_I32P), ax, n2.ctypes.data_as(_I32P), q.ctypes.data_as(_I32P),
                      _dptr(g.view(np.float64)))
    ps = "".join(paulis).encode()
    co = np.ascontiguousarray(coeffs, dtype=np.float64)
    h = tnsim_hamiltonian(len(paulis), ps, _dptr(co))
    e = C.c_double(0.0)
    grad = np.zeros(max(int(sum(n * len(a) for a in axes)), 1))
    _check(lib.tnsim_grad(C.byref(c), _dptr(th), C.byref(h), int(dtype),
                          C.byref(params) if params is not None else None, _P(int(stream)) if stream else None,
                          C.byref(e), _dptr(grad)))
    out, off = [], 0
    for a in axes:
        k = n * len(a)
        out.append(grad[off:off + k].reshape(n, len(a)).copy())
        off += k
    return e.value, out


def tnsim_last_stats(h) -> dict:
    st = tnsim_stats()
    _check(lib.tnsim_last_stats(h, C.byref(st)))
    return {k: getattr(st, k) for k, _ in tnsim_stats._fields_}


def tnsim_profile_enable(h, on: bool = True):
    _check(lib.tnsim_profile_enable(h, int(bool(on))))


def tnsim_profile_read(h) -> dict:
    """{kernel class: (total ms, launches)} since the last read."""
    ms = np.zeros(len(TNSIM_K_NAMES), dtype=np.float64)
    n = np.zeros(len(TNSIM_K_NAMES), dtype=np.int64)
    _check(lib.tnsim_profile_read(h, _dptr(ms), n.ctypes.data_as(_I64P)))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(TNSIM_K_NAMES)}


def tnsim_two_site_update_noalloc(site_a: int, cap_a: int, site_b: int, cap_b: int, chi_l: int,
                                  chi_m: int, chi_r: int, g4x4, chi_max: int, cutoff: float = 0.0,
                                  renormalize: bool = True, stream=None):
    """One complex64 two-qubit update on caller-owned device buffers (raw pointers),
    using the library's fixed scratch array.  Returns (k, eps, kept singular values)."""
    g = np.ascontiguousarray(g4x4, dtype=np.complex128).reshape(4, 4).view(np.float64)
    k = C.c_int32(0)
    eps = C.c_double(0.0)
    s = np.zeros(chi_max, dtype=np.float64)
    _check(lib.tnsim_two_site_update_noalloc(_P(site_a), int(cap_a), _P(site_b), int(cap_b), int(chi_l),
                                             int(chi_m), int(chi_r), _dptr(g), int(chi_max), float(cutoff),
                                             int(bool(renormalize)), _P(int(stream)) if stream else None,
                                             C.byref(k), C.byref(eps), _dptr(s)))
    return k.value, eps.value, s[: k.value].copy()


def tnsim_plan_create(handles, layers):
    """layers[i] = (q, g4_dev, u1_dev) for state i: host pair list and device pointers
    (ints; u1_dev may be 0).  Returns the plan handle."""
    n = len(handles)
    hs = (_P * n)(*[h.value if isinstance(h, _P) else h for h in handles])
    n2 = np.zeros(n, dtype=np.int32)
    qp = (_I32P * n)()
    gp = (_P * n)()
    up = (_P * n)()
    keep = []
    for i, (q, g, u) in enumerate(layers):
        q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1)
        keep.append(q)
        n2[i] = q.shape[0]
        qp[i] = q.ctypes.data_as(_I32P)
        gp[i] = g or None
        up[i] = u or None
    out = _P()
    _check(lib.tnsim_plan_create(hs, n, n2.ctypes.data_as(_I32P), qp, gp, up, C.byref(out)))
    return out


def tnsim_plan_launch(plan):
    _check(lib.tnsim_plan_launch(plan))


def tnsim_plan_destroy(plan):
    _check(lib.tnsim_plan_destroy(plan))


def tnsim_graph_create(plans):
    arr = (_P * len(plans))(*[p.value for p in plans])
    out = _P()
    _check(lib.tnsim_graph_create(arr, len(plans), C.byref(out)))
    return out


def tnsim_graph_launch(graph):
    _check(lib.tnsim_graph_launch(graph))


def tnsim_graph_destroy(graph):
    _check(lib.tnsim_graph_destroy(graph))


class MPS:
    """Owning wrapper of a tnsim_mps handle (argument marshalling only)."""

    def __init__(self, n_qubits: int, dtype: int = TNSIM_C64, chi_max: int = 64, cutoff: float = 0.0,
                 renormalize: bool = True, max_sweeps: int = 0, jacobi_tol: float = 0.0,
                 schedule: int = TNSIM_SCHED_BATCHED, gemm: int = TNSIM_GEMM_FP32, stream=None,
                 form: int = TNSIM_FORM_PAPER):
        p = tnsim_params_default(dtype)
        p.chi_max, p.cutoff, p.renormalize = int(chi_max), float(cutoff), int(bool(renormalize))
        p.max_sweeps, p.jacobi_tol, p.schedule = int(max_sweeps), float(jacobi_tol), int(schedule)
        p.gemm, p.form = int(gemm), int(form)
        self.n = int(n_qubits)
        self.dtype = dtype
        self.params = p
        self.h = tnsim_mps_create(n_qubits, dtype, p, stream)

    def close(self):
        if self.h is not None and self.h.value:
            tnsim_mps_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_layer(self, layer):
        return tnsim_apply_layer(self.h, layer.pairs, layer.g4, layer.u1)

    def run(self, circuit):
        return [self.apply_layer(l) for l in circuit.layers]

    def apply_circuit(self, ops):
        return tnsim_apply_circuit(self.h, ops)

    def sample(self, n_shots: int, seed: int = 0):
        """n_shots bitstrings; the uniforms are drawn on the host from numpy's PCG64(seed)."""
        u = np.random.default_rng(seed).random((int(n_shots), self.n))
        return tnsim_sample(self.h, u)[0]

    def bond_dims(self):
        return tnsim_bond_dims(self.h, self.n)

    def spectrum(self, bond):
        return tnsim_bond_spectrum(self.h, bond, self.params.chi_max)

    def export_sites(self):
        return tnsim_export_sites(self.h, self.n)

    def import_sites(self, sites):
        tnsim_import_sites(self.h, sites)

    def amplitudes(self, bits):
        return tnsim_amplitudes(self.h, bits)

    def expect_pauli(self, paulis):
        return tnsim_expect_pauli(self.h, paulis)

    def sync(self):
        tnsim_sync(self.h)

    def stats(self):
        return tnsim_last_stats(self.h)
