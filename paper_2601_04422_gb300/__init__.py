"""GB300 (sm_103a) MPS two-qubit-gate library: Python binding of libtnsim.so.

The compute path is the CUDA library built from ``csrc/`` (see ``include/tnsim.h``
for the C ABI).  This package only marshals arguments; importing it fails loudly
when the library has not been built -- there is no CPU fallback.
"""
from ._abi import (  # noqa: F401
    TNSIM_C64, TNSIM_C128, TNSIM_SCHED_BATCHED, TNSIM_SCHED_PLAIN, TNSIM_GEMM_FP32, TNSIM_GEMM_FP32_3M,
    TNSIM_GEMM_TF32X3, TNSIM_GEMM_BF16X3, TNSIM_FORM_PAPER, TNSIM_FORM_CANONICAL, TNSIM_OK, TNSIM_EINVAL,
    TNSIM_ENOMEM, TNSIM_ECUDA, TNSIM_ENOCONV, TNSIM_ETIMEOUT, TNSIM_EUNSUPPORTED,
    TnsimError, TnsimConvergenceWarning, lib, lib_path, exported_symbols,
    tnsim_params, tnsim_params_default, tnsim_mps_create, tnsim_mps_destroy, tnsim_apply_layer,
    tnsim_apply_layer_device, tnsim_apply_layers_batched, tnsim_sync, tnsim_bond_dims,
    tnsim_bond_spectrum, tnsim_export_sites, tnsim_import_sites, tnsim_amplitudes,
    tnsim_expect_pauli, tnsim_grad, tnsim_circuit, tnsim_hamiltonian, tnsim_last_stats, tnsim_last_error, tnsim_version,
    tnsim_stats, tnsim_profile_enable, tnsim_profile_read, TNSIM_K_NAMES,
    tnsim_two_site_update_noalloc, tnsim_plan_create, tnsim_plan_launch, tnsim_plan_destroy,
    tnsim_graph_create, tnsim_graph_launch, tnsim_graph_destroy, tnsim_apply_circuit,
    tnsim_circuit_layerize, tnsim_sample, tnsim_set_jacobi_config, tnsim_autotune, TNSIM_JACOBI_CONFIGS,
    tnsim_set_wait_limits, tnsim_set_device_memory_cap, tnsim_device_bytes_held,
    MPS,
)
