"""The allocation-free pipeline entry point (fft2_filter_ifft2_noalloc).

Some callers cannot allocate device memory while they run (inside CUDA
graph capture, in hosts that own every allocation, in loops that must not
block on cudaMalloc).  This entry point serves them with a fixed scratch
array inside the library.  Its output must match the plan-based entry point
fft2_filter_ifft2 within the pipeline tolerance, call after call, with the
shared scratch carrying over between calls.  The file is named to be
collected last.
"""

import ctypes

import numpy as np
import pytest

from paper_cs_0103001_gb300 import synth
from tests.gpu_util import max_rel_l2, tol_fp32

pytestmark = pytest.mark.gpu


def _noalloc(nat, img, H, h_stride, out):
    import torch

    rows, cols = img.shape[-2:]
    batch = img.numel() // (rows * cols)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return nat.lib.fft2_filter_ifft2_noalloc(rows, cols, batch, ctypes.c_void_p(img.data_ptr()),
                                             ctypes.c_void_p(H.data_ptr()), h_stride,
                                             ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_plan_entry_point():
    import torch

    import paper_cs_0103001_gb300 as gb
    from paper_cs_0103001_gb300 import _native as nat

    cases = [
        (512, 1024, 2, False),   # two images, shared filter
        (512, 1024, 2, False),   # same shape again: scratch reused as left
        (2048, 2048, 1, False),  # largest accepted image; twiddles regenerated
        (256, 128, 3, True),     # one filter per image
    ]
    for i, (rows, cols, batch, per_image) in enumerate(cases):
        img = torch.from_numpy(np.stack([synth.sky(rows, cols, 30, 20, i, b) for b in range(batch)])).cuda()
        if per_image:
            H = torch.from_numpy(np.stack([synth.random_filter(rows, cols, 21, i, b) for b in range(batch)])).cuda()
        else:
            H = torch.from_numpy(synth.random_filter(rows, cols, 21, i)).cuda()
        ref = gb.fft2_filter_ifft2(img, H)
        out = torch.full_like(img, float("nan"))
        rc = _noalloc(nat, img, H, rows * cols if per_image else 0, out)
        assert rc == nat.OK, nat.lib.gbfft_status_string(rc)
        torch.cuda.synchronize()
        assert max_rel_l2(out.cpu().numpy(), ref.cpu().numpy(), axes=(1, 2)) <= tol_fp32(rows * cols)


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    img = torch.zeros(16, 16, device="cuda")
    big = ctypes.c_void_p(img.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert nat.lib.fft2_filter_ifft2_noalloc(4096, 2048, 1, big, big, 0, big, s) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_filter_ifft2_noalloc(1000, 16, 1, big, big, 0, big, s) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_filter_ifft2_noalloc(16, 16, 1, None, big, 0, big, s) == nat.ERR_NULL
    odd = ctypes.c_void_p(img.data_ptr() + 4)
    assert nat.lib.fft2_filter_ifft2_noalloc(16, 16, 1, odd, big, 0, big, s) == nat.ERR_MISALIGNED
