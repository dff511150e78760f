"""ctypes binding of libgbfft.so (the C ABI in include/gbfft.h).

Argument marshalling only: every transform runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or fails to load,
importing this module raises.
"""

from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# GBFFT_CHECKED=1 loads the index-checking build (built by build.build(checked=True))
CHECKED = os.environ.get("GBFFT_CHECKED", "") not in ("", "0")
LIB_PATH = os.path.join(_PKG, "libgbfft_checked.so" if CHECKED else "libgbfft.so")

# gbfft_dtype
C64 = 1
C128 = 2

# gbfft_status
OK = 0
ERR_NULL = -1
ERR_INVALID_SIZE = -2
ERR_DTYPE = -3
ERR_MISALIGNED = -4
ERR_WORKSPACE = -5
ERR_UNSUPPORTED = -6
ERR_CUDA = -7
ERR_TIMEOUT = -8
ERR_INVALID_VALUE = -9

# gbfft_option
OPT_SCALE_CONVENTION = 1
OPT_H_BATCH_STRIDE = 2
OPT_PRECISION = 3
OPT_IMAGES_PER_CHUNK = 4
OPT_PROFILE = 5
OPT_ENABLE_BACKWARD = 6
OPT_BLOCKS_PER_SM = 7
OPT_USE_GRAPH = 8
OPT_ONCHIP = 9
OPT_COLUMN_FORM = 10
OPT_BATCH_FORM = 11
OPT_FOURSTEP_PASSES = 12

# gbfft_filter_kind
FILTER_GAUSSIAN = 1
FILTER_BUTTERWORTH = 2
FILTER_DISC = 3

# gbfft_stage
STAGES = ("fft1d", "fourstep_a", "fourstep_b", "rows_fwd", "cols_filter", "rows_inv", "cols_grad", "twiddles",
          "graph", "filter_prep", "onchip", "spectrum", "fft1d_cluster")

# every exported symbol with (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
SIGNATURES = {
    "fft_plan_create": (_INT, [_I64, _I64, _INT, ctypes.POINTER(_P)]),
    "fft2_plan_create": (_INT, [_I64, _I64, _I64, _INT, ctypes.POINTER(_P)]),
    "fft_plan_set_option": (_INT, [_P, _INT, _I64]),
    "fft_plan_workspace_bytes": (_INT, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "fft_plan_bind_workspace": (_INT, [_P, _P, ctypes.c_size_t, _P]),
    "fft_forward": (_INT, [_P, _P, _P, _P]),
    "fft_inverse": (_INT, [_P, _P, _P, _P]),
    "fft2_filter_ifft2": (_INT, [_P, _P, _P, _P, _P]),
    "fft2_filter_prepare": (_INT, [_P, _P, _P]),
    "fft2_filter_ifft2_prepared": (_INT, [_P, _P, _P, _P]),
    "fft2_filter_ifft2_padded": (_INT, [_P, _P, _I64, _I64, _P, _P, _P]),
    "fft2_spectrum": (_INT, [_P, _P, _I64, _I64, _P, _P]),
    "fft2_filter_ifft2_analytic": (_INT, [_P, _P, _INT, ctypes.c_double, ctypes.c_double, _P, _P]),
    "gbfft_device_status": (_INT, [_P]),
    "gbfft_plan_check_guards": (_INT, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "gbfft_checked_take": (_INT, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "gbfft_selftest_wait_timeout": (_INT, [_P, _I64, _P]),
    "gbfft_selftest_corrupt_work_item": (_INT, [_P, _INT, _I64, _INT, _INT]),
    "gbfft_selftest_launch_config": (_INT, [_P]),
    "fft2_filter_ifft2_backward": (_INT, [_P, _P, _P, _P, _P, _P, _P]),
    "fft_plan_destroy": (_INT, [_P]),
    "fft2_batched_plan_create": (_INT, [_INT, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_P)]),
    "fft2_filter_ifft2_batched": (_INT, [_P, _P, _P]),
    "fft_plan_autotune": (_INT, [_P, _P, _P]),
    "fft_plan_get_option": (_INT, [_P, _INT, ctypes.POINTER(_I64)]),
    "fft2_filter_ifft2_noalloc": (_INT, [_I64, _I64, _I64, _P, _P, _I64, _P, _P]),
    "fft2_slab_plan_create": (_INT, [_I64, _I64, _INT, _INT, ctypes.POINTER(_P)]),
    "fft2_slab_exchange_elems": (_INT, [_P, ctypes.POINTER(_I64)]),
    "fft2_slab_rows_forward": (_INT, [_P, _P, _P, _P]),
    "fft2_slab_columns": (_INT, [_P, _P, _P, _P]),
    "fft2_slab_rows_inverse": (_INT, [_P, _P, _P, _P]),
    "gbfft_status_string": (ctypes.c_char_p, [_INT]),
    "gbfft_last_cuda_error": (_INT, []),
    "gbfft_plan_profile_read": (_INT, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64), _INT]),
    "gbfft_version": (_INT, []),
    "gbfft_measure_fma_peak": (_INT, [_INT, ctypes.POINTER(ctypes.c_double), _P]),
}


class GbfftError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = lib.gbfft_status_string(status).decode() if lib is not None else str(status)
        extra = f" (cudaError {lib.gbfft_last_cuda_error()})" if status == ERR_CUDA else ""
        super().__init__(f"{fn} failed: {msg} [{status}]{extra}")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libgbfft.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()'; the checked build: "
            "paper_cs_0103001_gb300.build.build(checked=True))"
        )
    so = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


lib = _load()


def check(fn: str, status: int) -> None:
    if status != OK:
        raise GbfftError(fn, status)


def call(fn: str, *args) -> None:
    check(fn, getattr(lib, fn)(*args))
