"""The C-ABI library builds, loads and exports every entry point its header declares.

CPU only: no entry point that touches the GPU is called here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    return T


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tnsim_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(T):
    declared = _declared()
    assert "tnsim_apply_layer" in declared and "tnsim_mps_create" in declared
    lib = ctypes.CDLL(T.lib_path)
    for name in declared:
        assert hasattr(lib, name), name
    assert set(T.exported_symbols()) <= set(declared)


def test_params_default_and_version(T):
    p = T.tnsim_params_default(T.TNSIM_C64)
    assert p.chi_max == 64 and p.cutoff == 0.0 and p.renormalize == 1 and p.schedule == 0 and p.form == 0
    assert "sm_103a" in T.tnsim_version()
    with pytest.raises(T.TnsimError):
        T.tnsim_params_default(7)


def test_params_struct_layout_matches_header(T):
    # offsets of the C struct (int32, double, int32, int32, double, int32, int32, int32) with
    # natural alignment
    P = T.tnsim_params
    assert P.cutoff.offset == 8 and P.renormalize.offset == 16 and P.max_sweeps.offset == 20
    assert P.jacobi_tol.offset == 24 and P.schedule.offset == 32 and P.gemm.offset == 36
    assert P.form.offset == 40 and ctypes.sizeof(P) == 48


def test_library_is_sm103a_only():
    """The build targets sm_103a and nothing else."""
    import __graft_entry__ as g
    b = g._build_module()
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
