"""The allocation-free pipeline entry point (fft2_filter_ifft2_noalloc).

Some callers cannot allocate device memory while they run: loops where a
cudaMalloc could block or synchronise the device, and plugins whose host
application owns every device allocation.  This entry point serves them with
a fixed scratch array inside the library.  Its output must match the
plan-based entry point fft2_filter_ifft2 and the FP64 oracle within the
pipeline tolerance, call after call, with the shared scratch carrying over
between calls.  The file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import oracle
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


def test_noalloc_matches_plan_entry_point_and_oracle():
    import torch

    import paper_cs_0103001_gb300 as gb
    from paper_cs_0103001_gb300 import _native as nat

    cases = [
        (512, 1024, 2, False),   # two images, shared filter
        (512, 1024, 2, False),   # same shape again: scratch reused as left
        (2048, 2048, 1, False),  # largest accepted image
        (8192, 512, 1, False),   # tall: columns of 8192 rows
        (256, 128, 3, True),     # one filter per image
        (512, 1024, 2, False),   # back to the first shape after others
    ]
    for i, (rows, cols, batch, per_image) in enumerate(cases):
        img_np = np.stack([synth.sky(rows, cols, 30, 20, i, b) for b in range(batch)])
        if per_image:
            H_np = np.stack([synth.random_filter(rows, cols, 21, i, b) for b in range(batch)])
        else:
            H_np = synth.random_filter(rows, cols, 21, i)
        img, H = torch.from_numpy(img_np).cuda(), torch.from_numpy(H_np).cuda()
        ref = gb.fft2_filter_ifft2(img, H)
        out = torch.full_like(img, float("nan"))
        rc = _noalloc(nat, img, H, rows * cols if per_image else 0, out)
        assert rc == nat.OK, nat.lib.gbfft_status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = tol_fp32(rows * cols)
        assert max_rel_l2(got, ref.cpu().numpy(), axes=(1, 2)) <= tol
        want = np.stack([oracle.pipeline(img_np[b], H_np[b] if per_image else H_np) for b in range(batch)])
        assert max_rel_l2(got, want, axes=(1, 2)) <= tol


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
