"""GPU parity of the pipeline with analytic filters computed in the column
pass (Gaussian, Butterworth, the disc of Eq. filtro) against the FP64 oracle
run with the same filter written out as an array."""

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import max_rel_l2, rel_l2, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch

    import paper_cs_0103001_gb300 as gb

    assert torch.cuda.is_available()
    return gb


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [(16, 16), (64, 256), (256, 64), (512, 512), (1024, 2048), (4096, 4096), (8192, 16)]


@pytest.mark.parametrize("rows,cols", SHAPES)
def test_gaussian(gb, rows, cols):
    from paper_cs_0103001_gb300 import _native as nat

    img = synth.sky(rows, cols, max(1, rows * cols // 4000), 60, rows, cols)
    sigma = max(2.0, min(rows, cols) / 16)
    got = gb.fft2_filter_ifft2_analytic(_cuda(img), nat.FILTER_GAUSSIAN, sigma).cpu().numpy()
    want = oracle.pipeline(img, synth.gaussian_lowpass(rows, cols, sigma))
    assert rel_l2(got, want) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("rows,cols", SHAPES)
def test_butterworth(gb, rows, cols):
    from paper_cs_0103001_gb300 import _native as nat

    img = synth.sky(rows, cols, max(1, rows * cols // 4000), 61, rows, cols)
    d0 = 0.1 * min(rows, cols) / 2.0
    got = gb.fft2_filter_ifft2_analytic(_cuda(img), nat.FILTER_BUTTERWORTH, 4, d0).cpu().numpy()
    want = oracle.pipeline(img, synth.butterworth_lowpass(rows, cols, 4, 0.1))
    assert rel_l2(got, want) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("rows,cols,b", [(512, 512, 340.0), (256, 512, 170.0), (64, 64, 20.5), (16, 32, 0.0)])
def test_disc(gb, rows, cols, b):
    """Eq. filtro, ties at distance exactly b included (340^2 = 204^2 + 272^2)."""
    from paper_cs_0103001_gb300 import _native as nat

    img = synth.sky(rows, cols, max(1, rows * cols // 4000), 62, rows, cols)
    H = synth.disc_filter(rows, cols, b)
    got = gb.fft2_filter_ifft2_analytic(_cuda(img), nat.FILTER_DISC, b).cpu().numpy()
    assert rel_l2(got, oracle.pipeline(img, H)) <= tol_fp32(rows * cols)
    expl = gb.fft2_filter_ifft2(_cuda(img), _cuda(H)).cpu().numpy()
    assert rel_l2(got, expl) <= 2 * tol_fp32(rows * cols)


def test_batch_and_bad_parameters(gb):
    from paper_cs_0103001_gb300 import _native as nat

    rows, cols, B = 128, 256, 5
    img = np.stack([synth.sky(rows, cols, 20, 63, b) for b in range(B)])
    plan = gb.Plan2D(rows, cols, B, "cuda", {nat.OPT_IMAGES_PER_CHUNK: 2})
    got = plan.filter_analytic(_cuda(img), nat.FILTER_GAUSSIAN, 9.0).cpu().numpy()
    want = oracle.pipeline(img, synth.gaussian_lowpass(rows, cols, 9.0))
    assert max_rel_l2(got, want, axes=(1, 2)) <= tol_fp32(rows * cols)
    t = _cuda(img)
    for kind, p0, p1 in ((0, 1.0, 0.0), (4, 1.0, 0.0), (nat.FILTER_GAUSSIAN, 0.0, 0.0),
                         (nat.FILTER_BUTTERWORTH, 2.5, 10.0), (nat.FILTER_BUTTERWORTH, 4, 0.0),
                         (nat.FILTER_DISC, -1.0, 0.0)):
        with pytest.raises(RuntimeError):
            plan.filter_analytic(t, kind, p0, p1)
