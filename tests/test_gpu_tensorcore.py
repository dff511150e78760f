"""The 2D pipeline with its radix-16 passes as split-precision DFT-matrix
products on the tensor cores, against the FP64 oracle: warp-level mma.sync
(GBFFT_OPT_PRECISION 1 and 2) and the fifth-generation tcgen05.mma with
accumulators in tensor memory (3, 4: BF16 in 2 or 3 parts; 5: TF32 in 2).

Two BF16 parts per operand (three products) keep about 16 significant bits
per pass, so that variant is held to a looser bound than FP32 and its error
is recorded; three parts (six products) keep about 24 bits and meet the FP32
tolerance."""

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import rel_l2, tol_fp32

pytestmark = pytest.mark.gpu


def _run(rows, cols, precision, seed):
    import torch

    import paper_cs_0103001_gb300 as gb
    from paper_cs_0103001_gb300 import _native as nat

    img = synth.sky(rows, cols, max(5, rows * cols // 4000), seed)
    H = synth.butterworth_lowpass(rows, cols, 4, 0.1)
    plan = gb.Plan2D(rows, cols, 1, "cuda", {nat.OPT_PRECISION: precision})
    out = plan.filter(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda())
    return rel_l2(out.cpu().numpy(), oracle.pipeline(img, H))


@pytest.mark.parametrize("rows,cols", [(512, 512), (1024, 512), (512, 2048), (4096, 4096)])
def test_split_bf16_pipeline(rows, cols):
    e32 = _run(rows, cols, 0, 50)
    e2 = _run(rows, cols, 1, 50)
    e3 = _run(rows, cols, 2, 50)
    print(f"{rows}x{cols}: fp32 {e32:.2e}  bf16x2 (3 products) {e2:.2e}  bf16x3 (6 products) {e3:.2e}")
    assert e3 <= tol_fp32(rows * cols)
    assert e2 <= 50 * tol_fp32(rows * cols)
    assert e3 <= e2


@pytest.mark.parametrize("rows,cols", [(512, 512), (1024, 512), (512, 2048), (2048, 1024), (4096, 4096)])
def test_tcgen05_pipeline(rows, cols):
    """tcgen05 passes: six BF16 products and three TF32 products meet the FP32
    tolerance; three BF16 products keep about 16 bits per pass, as on mma.sync."""
    e32 = _run(rows, cols, 0, 51)
    e3 = _run(rows, cols, 3, 51)
    e4 = _run(rows, cols, 4, 51)
    e5 = _run(rows, cols, 5, 51)
    print(f"{rows}x{cols}: fp32 {e32:.2e}  tcgen05 bf16x2 {e3:.2e}  bf16x3 {e4:.2e}  tf32x2 {e5:.2e}")
    assert e4 <= tol_fp32(rows * cols)
    assert e5 <= tol_fp32(rows * cols)
    assert e3 <= 50 * tol_fp32(rows * cols)
    assert e4 <= e3


def test_unsupported_sizes_are_refused():
    import ctypes

    from paper_cs_0103001_gb300 import _native as nat

    h = ctypes.c_void_p()
    assert nat.lib.fft2_plan_create(256, 512, 1, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_PRECISION, 1) == nat.ERR_UNSUPPORTED
    nat.lib.fft_plan_destroy(h)
    assert nat.lib.fft_plan_create(1024, 4, 1, ctypes.byref(h)) == nat.OK
    assert nat.lib.fft_plan_set_option(h, nat.OPT_PRECISION, 2) == nat.ERR_UNSUPPORTED
    nat.lib.fft_plan_destroy(h)
