"""Failure paths on the GPU without a GPU fault: a launch the CUDA runtime
refuses (a block of 2048 threads) is reported as a status and leaves the
context usable; a corrupted work list of a batched plan is refused when the
plan binds; and the NVTX stage ranges (GBFFT_NVTX=1) change no result."""

import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import max_rel_l2, tol_fp32

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_refused_launch_is_reported_and_the_context_stays_usable():
    import torch

    import paper_cs_0103001_gb300 as gb
    from paper_cs_0103001_gb300 import _native as nat
    from paper_cs_0103001_gb300.api import _stream_handle

    st = nat.lib.gbfft_selftest_launch_config(_stream_handle(torch.device("cuda")))
    assert st == nat.ERR_CUDA
    # the runtime's refusal: cudaErrorInvalidValue (1, what CUDA 13 returns for a
    # block larger than 1024 threads) or cudaErrorInvalidConfiguration (9)
    assert nat.lib.gbfft_last_cuda_error() in (1, 9)
    x = synth.complex_uniform((3, 4096), 60)
    y = gb.fft(torch.from_numpy(x).cuda()).cpu().numpy()
    assert max_rel_l2(y, oracle.fft(x.astype(np.complex128)), axes=-1) <= tol_fp32(4096)


def test_corrupted_work_item_is_refused_at_bind():
    import ctypes

    import torch

    from paper_cs_0103001_gb300 import _native as nat
    from paper_cs_0103001_gb300.api import _stream_handle

    shapes = [(128, 128), (512, 256)]
    rows = (ctypes.c_int64 * 2)(*[r for r, _ in shapes])
    cols = (ctypes.c_int64 * 2)(*[c for _, c in shapes])
    h = ctypes.c_void_p()
    assert nat.lib.fft2_batched_plan_create(2, rows, cols, ctypes.byref(h)) == nat.OK
    ws = ctypes.c_size_t()
    assert nat.lib.fft_plan_workspace_bytes(h, ctypes.byref(ws)) == nat.OK
    buf = torch.empty(ws.value, dtype=torch.uint8, device="cuda")
    s = _stream_handle(torch.device("cuda"))
    assert nat.lib.fft_plan_bind_workspace(h, ctypes.c_void_p(buf.data_ptr()), ws.value, s) == nat.OK
    assert nat.lib.gbfft_selftest_corrupt_work_item(h, 1, 0, 7, 0) == nat.OK
    assert nat.lib.fft_plan_bind_workspace(h, ctypes.c_void_p(buf.data_ptr()), ws.value, s) == nat.ERR_INVALID_VALUE
    ptrs = torch.zeros(2, 3, dtype=torch.int64, device="cuda")
    assert nat.lib.fft2_filter_ifft2_batched(h, ctypes.c_void_p(ptrs.data_ptr()), s) == nat.ERR_WORKSPACE
    assert nat.lib.fft_plan_destroy(h) == nat.OK
    torch.cuda.synchronize()


def test_nvtx_ranges_change_no_result():
    code = (
        "import numpy as np, torch, oracle\n"
        "import paper_cs_0103001_gb300 as gb\n"
        "from paper_cs_0103001_gb300 import synth\n"
        "img = synth.sky(512, 1024, 100, 61)\n"
        "H = synth.gaussian_lowpass(512, 1024, 40.0)\n"
        "out = gb.fft2_filter_ifft2(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()).cpu().numpy()\n"
        "ref = oracle.pipeline(img, H)\n"
        "print(float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))\n"
    )
    env = dict(os.environ, GBFFT_NVTX="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert float(r.stdout.strip().splitlines()[-1]) <= tol_fp32(512 * 1024)
