"""Host-side checks of the C ABI (no GPU needed).

The library must load without a GPU, export every function that
include/gbfft.h declares, and reject bad arguments with the documented
status codes before touching CUDA.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbfft.h")


@pytest.fixture(scope="module")
def nat():
    import __graft_entry__ as g

    g._build_module().build()
    from paper_cs_0103001_gb300 import _native

    return _native


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fft_plan_create", "fft_forward", "fft_inverse", "fft2_filter_ifft2", "fft_plan_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(nat):
    so = ctypes.CDLL(nat.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, f"declared but not exported: {missing}"
    # and the binding knows each of them
    assert set(declared_functions()) <= set(nat.SIGNATURES)


def _plan(nat, n=1024, batch=2, dtype=1):
    h = ctypes.c_void_p()
    rc = nat.lib.fft_plan_create(n, batch, dtype, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("n", [0, 1, 3, 1000, 1 << 25, -4])
def test_plan_rejects_bad_lengths(nat, n):
    rc, h = _plan(nat, n=n)
    assert rc == nat.ERR_INVALID_SIZE and not h.value


def test_plan_rejects_bad_batch_and_dtype(nat):
    assert _plan(nat, batch=0)[0] == nat.ERR_INVALID_SIZE
    assert _plan(nat, dtype=7)[0] == nat.ERR_DTYPE
    assert nat.lib.fft_plan_create(8, 1, 1, None) == nat.ERR_NULL
    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(100, 64, 1, 1, ctypes.byref(h)) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_plan_create(64, 64, 1, 2, ctypes.byref(h)) == nat.ERR_DTYPE
    assert nat.lib.fft2_plan_create(1 << 14, 64, 1, 1, ctypes.byref(h)) == nat.ERR_INVALID_SIZE


def test_workspace_and_pointer_checks(nat):
    rc, h = _plan(nat, n=4096, batch=3)
    assert rc == nat.OK
    b = ctypes.c_size_t()
    assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(b)) == nat.OK
    assert b.value >= 4096 * 8
    fake = ctypes.c_void_p(1 << 20)
    # no workspace bound yet
    assert nat.lib.fft_forward(h, fake, fake, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_bind_workspace(h, None, b.value, None) == nat.ERR_NULL
    assert nat.lib.fft_plan_bind_workspace(h, fake, b.value - 1, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_bind_workspace(h, ctypes.c_void_p((1 << 20) + 16), b.value, None) == nat.ERR_MISALIGNED
    assert nat.lib.fft_plan_destroy(h) == nat.OK
    assert nat.lib.fft_plan_destroy(None) == nat.ERR_NULL


def test_options(nat):
    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(256, 512, 4, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_SCALE_CONVENTION, 1) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_SCALE_CONVENTION, 2) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft_plan_set_option(h, nat.OPT_H_BATCH_STRIDE, 256 * 512) == nat.OK
    assert nat.lib.fft_plan_set_option(h, 999, 0) == nat.ERR_INVALID_VALUE
    b1, b2 = ctypes.c_size_t(), ctypes.c_size_t()
    assert nat.lib.fft_plan_set_option(h, nat.OPT_IMAGES_PER_CHUNK, 1) == nat.OK
    nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(b1))
    assert nat.lib.fft_plan_set_option(h, nat.OPT_IMAGES_PER_CHUNK, 4) == nat.OK
    nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(b2))
    assert b2.value > b1.value >= 256 * 256 * 8
    fake = ctypes.c_void_p(1 << 20)
    # 1D calls on a 2D plan are a kind mismatch (checked after the workspace)
    assert nat.lib.fft_forward(h, fake, fake, None) == nat.ERR_WORKSPACE
    nat.lib.fft_plan_destroy(h)


def test_status_strings(nat):
    for code in range(-9, 1):
        assert nat.lib.gbfft_status_string(code)
    assert nat.lib.gbfft_version() >= 100


def test_padded_and_spectrum_entry_checks(nat):
    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(512, 512, 1, 1, ctypes.byref(h)) == nat.OK
    fake = ctypes.c_void_p(1 << 20)
    assert nat.lib.fft2_filter_ifft2_padded(None, fake, 460, 506, fake, fake, None) == nat.ERR_NULL
    assert nat.lib.fft2_spectrum(None, fake, 460, 506, fake, None) == nat.ERR_NULL
    # no workspace bound yet
    assert nat.lib.fft2_filter_ifft2_padded(h, fake, 460, 506, fake, fake, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft2_spectrum(h, fake, 460, 506, fake, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_analytic_entry_checks(nat):
    fake = ctypes.c_void_p(1 << 20)
    assert nat.lib.fft2_filter_ifft2_analytic(None, fake, nat.FILTER_GAUSSIAN, 3.0, 0.0, fake, None) == nat.ERR_NULL
    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(64, 64, 1, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft2_filter_ifft2_analytic(h, fake, nat.FILTER_GAUSSIAN, 3.0, 0.0, fake, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_device_status_checks(nat):
    assert nat.lib.gbfft_device_status(None) == nat.ERR_NULL
    rc, h = _plan(nat, n=1 << 20, batch=1)
    assert rc == nat.OK
    assert nat.lib.gbfft_device_status(h) == nat.ERR_WORKSPACE  # nothing bound yet
    assert nat.lib.gbfft_selftest_wait_timeout(None, 1, None) == nat.ERR_NULL
    assert nat.lib.gbfft_selftest_wait_timeout(h, 16, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_slab_plan_validation_without_gpu(nat):
    h = ctypes.c_void_p()
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 3, 0, ctypes.byref(h)) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_slab_plan_create(128, 128, 2, 0, ctypes.byref(h)) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 2, 5, ctypes.byref(h)) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 2, 1, None) == nat.ERR_NULL
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 2, 1, ctypes.byref(h)) == nat.OK and h.value
    n = ctypes.c_int64()
    assert nat.lib.fft2_slab_exchange_elems(h, ctypes.byref(n)) == nat.OK
    assert n.value == 2048 * 2048
    ws = ctypes.c_size_t()
    assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(ws)) == nat.OK and ws.value > 0
    # no workspace bound yet: every step refuses before touching CUDA
    buf = ctypes.c_void_p(256)
    assert nat.lib.fft2_slab_rows_forward(h, buf, buf, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft2_slab_columns(h, buf, buf, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft2_slab_rows_inverse(h, buf, buf, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_corrupted_work_list_is_refused_before_the_gpu(nat):
    """A batched plan's work items index images and blocks unchecked on the
    GPU; binding checks every item on the host first.  A corrupted item
    (image or block out of range) makes the bind return
    GBFFT_ERR_INVALID_VALUE without a CUDA call (this test has no GPU)."""
    shapes = [(64, 128), (256, 256), (1024, 512)]
    rows = (ctypes.c_int64 * 3)(*[r for r, _ in shapes])
    cols = (ctypes.c_int64 * 3)(*[c for _, c in shapes])
    ws = ctypes.c_size_t()
    fake = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced: the bind stops before CUDA
    for stage, img, bx in [(0, 3, 0), (1, -1, 0), (2, 0, 1 << 20), (3, 2, -5), (0, 0, 32)]:
        h = ctypes.c_void_p()
        assert nat.lib.fft2_batched_plan_create(3, rows, cols, ctypes.byref(h)) == nat.OK
        assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(ws)) == nat.OK
        assert nat.lib.gbfft_selftest_corrupt_work_item(h, stage, 0, img, bx) == nat.OK
        assert nat.lib.fft_plan_bind_workspace(h, fake, ws.value, None) == nat.ERR_INVALID_VALUE
        # unbound: the pipeline refuses too
        assert nat.lib.fft2_filter_ifft2_batched(h, fake, None) == nat.ERR_WORKSPACE
        assert nat.lib.fft_plan_destroy(h) == nat.OK
    h = ctypes.c_void_p()
    assert nat.lib.fft2_batched_plan_create(3, rows, cols, ctypes.byref(h)) == nat.OK
    assert nat.lib.gbfft_selftest_corrupt_work_item(h, 4, 0, 0, 0) == nat.ERR_INVALID_VALUE
    assert nat.lib.gbfft_selftest_corrupt_work_item(h, 0, 1 << 30, 0, 0) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft_plan_destroy(h) == nat.OK
    assert nat.lib.fft_plan_create(1024, 4, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.gbfft_selftest_corrupt_work_item(h, 0, 0, 0, 0) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_prepared_filter_entry_checks(nat):
    """The prepared-filter calls refuse, before any CUDA call, a null plan
    and an unbound one."""
    buf = ctypes.c_void_p(256)
    assert nat.lib.fft2_filter_prepare(None, buf, None) == nat.ERR_NULL
    assert nat.lib.fft2_filter_ifft2_prepared(None, buf, buf, None) == nat.ERR_NULL
    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(256, 512, 1, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft2_filter_prepare(h, buf, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft2_filter_ifft2_prepared(h, buf, buf, None) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK


def test_fourstep_passes_option(nat):
    """GBFFT_OPT_FOURSTEP_PASSES: three passes by default for complex64 at
    2^24 only; 2 or 3 accepted on 1D plans, other values and other plans
    refused; the choice changes the workspace size."""
    h = ctypes.c_void_p()
    v = ctypes.c_int64()
    ws2, ws3 = ctypes.c_size_t(), ctypes.c_size_t()
    assert nat.lib.fft_plan_create(1 << 24, 2, nat.C64, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft_plan_get_option(h, nat.OPT_FOURSTEP_PASSES, ctypes.byref(v)) == nat.OK and v.value == 3
    assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(ws3)) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_FOURSTEP_PASSES, 2) == nat.OK
    assert nat.lib.fft_plan_get_option(h, nat.OPT_FOURSTEP_PASSES, ctypes.byref(v)) == nat.OK and v.value == 2
    assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(ws2)) == nat.OK and ws2.value != ws3.value
    assert nat.lib.fft_plan_set_option(h, nat.OPT_FOURSTEP_PASSES, 4) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft_plan_destroy(h) == nat.OK
    for n, dt in ((1 << 20, nat.C64), (1 << 24, nat.C128)):
        assert nat.lib.fft_plan_create(n, 1, dt, ctypes.byref(h)) == nat.OK
        assert nat.lib.fft_plan_get_option(h, nat.OPT_FOURSTEP_PASSES, ctypes.byref(v)) == nat.OK and v.value == 2
        assert nat.lib.fft_plan_destroy(h) == nat.OK
    assert nat.lib.fft2_plan_create(256, 256, 1, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_FOURSTEP_PASSES, 3) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft_plan_destroy(h) == nat.OK
