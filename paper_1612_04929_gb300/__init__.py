"""GB300 (sm_103a) forward + exact-gradient evaluation of piecewise-constant quantum-control
costs (Leung, Abdelhafez, Koch, Schuster, arXiv:1612.04929).

The computation lives in the CUDA library built from ``csrc/`` (``build.py``); ``qoc`` is the
ctypes binding of its C ABI (``include/qoc.h``).
"""
from .qoc import (ABI_SYMBOLS, Batch, Context, QocError, QOCCost, cost, load, qoc_create, qoc_default_options,  # noqa: F401
                  qoc_destroy, qoc_evaluate_cost_and_grad, qoc_evaluate_batch, qoc_evaluate_device, qoc_evaluate_static, qoc_get_info,
                  qoc_last_error, qoc_get_profile, qoc_measure_fma_peak, qoc_reset_profile, qoc_set_ensemble, qoc_set_system, qoc_set_targets, qoc_status_string,
                  qoc_sync)
