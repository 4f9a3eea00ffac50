"""ctypes binding of libiqp_gb300.so (the C ABI of include/iqp.h).

Argument marshalling only. If the library is missing this raises: there is
no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiqp_gb300.so")
# The self-checked build (build.build(checks=True)) sits beside it; setting
# IQP_CHECKED_LIB=1 loads that one instead.
CHECKED_LIB_PATH = os.path.join(HERE, "libiqp_gb300_checked.so")
if os.environ.get("IQP_CHECKED_LIB") == "1":
    LIB_PATH = CHECKED_LIB_PATH

OK, ERR_ARG, ERR_ALIGN, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
FP32, SPLIT_BF16, SPARSE_FP32, LOWORDER_FP32 = 0, 1, 2, 3
OP_EXPVAL, OP_EXPVAL_GRAD, OP_MMD_LOSS, OP_MMD_LOSS_GRAD, OP_BITFLIP = 1, 2, 3, 4, 5
OP_EXPVAL_INDEP, OP_EXPVAL_INDEP_GRAD, OP_MMD_LOSS_INDEP, OP_MMD_LOSS_GRAD_INDEP = 6, 7, 8, 9
MMD_UNBIASED, MMD_SQRT, MMD_INDEP = 1, 2, 4

# Every symbol include/iqp.h declares, with (restype, argtypes).
_i64, _p, _int, _sz, _dbl = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
_MAT = [_p, _i64, _i64]
SIGNATURES = {
    "iqp_workspace_bytes": (_sz, [_int, _i64, _i64, _i64, _i64, _i64, _int]),
    "iqp_parity": (_int, [_i64] + _MAT + _MAT + [_p, _i64, _p]),
    "iqp_parity_gather": (_int, [_i64] + _MAT + _MAT + [_p, _i64, _p, _i64, _p, _p]),
    "iqp_parity_sum": (_int, [_i64] + _MAT + _MAT + [_p, _p]),
    "iqp_expval": (_int, [_i64] + _MAT * 3 + [_p, _int, _p, _p, _p, _sz, _p]),
    "iqp_expval_noalloc": (_int, [_i64] + _MAT * 3 + [_p, _int, _p, _p, _p]),
    "iqp_noalloc_read_status": (_int, [_p]),
    "iqp_expval_grad": (_int, [_i64] + _MAT * 3 + [_p, _p, _p, _int, _p, _p, _sz, _p]),
    "iqp_mmd_loss": (_int, [_i64] + _MAT * 4 + [_p, _int, _int, _p, _p, _sz, _p]),
    "iqp_mmd_loss_grad": (_int, [_i64] + _MAT * 4 + [_p, _int, _int, _p, _p, _p, _sz, _p]),
    "iqp_bitflip_expval": (_int, [_i64] + _MAT * 2 + [_p, _p, _p, _sz, _p]),
    "iqp_bitflip_grad": (_int, [_i64] + _MAT * 2 + [_p, _p, _p, _p, _sz, _p]),
    "iqp_expval_value_and_grad": (_int, [_i64] + _MAT * 3 + [_p, _p, _p, _int, _p, _p, _p, _p, _sz, _p]),
    "iqp_expval_keep_phi": (_int, [_i64] + _MAT * 3 + [_p, _int, _p, _p, _p, _i64, _p, _sz, _p]),
    "iqp_expval_grad_from_phi": (_int, [_i64] + _MAT * 3 + [_p, _p, _p, _int, _p, _i64, _p, _p, _sz, _p]),
    "iqp_expval_indep": (_int, [_i64] + _MAT * 3 + [_p, _p, _p, _p, _sz, _p]),
    "iqp_expval_indep_grad": (_int, [_i64] + _MAT * 3 + [_p, _p, _p, _p, _p, _sz, _p]),
    "iqp_expand_params": (_int, [_p, _i64, _p, _p, _i64, _p]),
    "iqp_reduce_params": (_int, [_p, _i64, _p, _i64, _p, _p]),
    "iqp_embed_bits": (_int, [_p, _i64, _i64, _p, _i64, _p, _i64, _i64, _p]),
    "iqp_uniform_bits": (_int, [ctypes.c_uint64, ctypes.c_uint64, _i64, _i64, _p, _i64, _p]),
    "iqp_bernoulli_bits": (_int, [ctypes.c_uint64, ctypes.c_uint64, _i64, _i64, _dbl, _p, _i64, _p]),
    "iqp_read_status": (_int, [_p, _sz, _p]),
    "iqp_selftest_timeout": (_int, [_p, _sz, _dbl, _p]),
    "iqp_status_string": (ctypes.c_char_p, [_int]),
    "iqp_launch_count": (ctypes.c_uint64, []),
    "iqp_tensor_path_available": (_int, []),
    "iqp_check_status": (ctypes.c_uint32, []),
    "iqp_checks_enabled": (_int, []),
    "iqp_profile_enable": (None, [_int]),
    "iqp_profile_reset": (None, []),
    "iqp_profile_query": (_int, [_int, _p, _p]),
}

KERNELS = ["parity", "parity_sum", "theta_split", "phase_fp32", "recompute_fp32", "grad_fp32", "phase_tc",
           "recompute_tc", "grad_tc", "finalize", "grad_reduce", "mmd_combine", "selftest", "bitflip",
           "phase_sparse", "grad_sparse", "variants", "rng", "loworder",
           "loworder_gemm"]

_lib = None


class IqpError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


def load() -> ctypes.CDLL:
    """Load the library (once). Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    try:
        return load().iqp_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return "unknown"


def check(status: int, what: str) -> None:
    if status != OK:
        raise IqpError(status, what)
