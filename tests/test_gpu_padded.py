"""GPU parity of Sec. 5's application path for images whose sides are not
powers of two (zero padding, filter, crop) and of the spectrum display
|fft2|, against the FP64 oracle, through the C ABI."""

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


@pytest.mark.parametrize("r,c,R,C", [(460, 506, 512, 512), (5, 6, 8, 8), (1, 1, 2, 2), (100, 37, 128, 64),
                                     (256, 255, 256, 256), (33, 1000, 64, 1024), (300, 17, 4096, 32),
                                     (64, 64, 64, 64)])
def test_padded_pipeline(gb, r, c, R, C):
    img = synth.sky(r, c, max(1, r * c // 2000), 50, r, c)
    H = synth.random_filter(R, C, 51, R, C)
    got = gb.fft2_filter_ifft2_padded(_cuda(img), _cuda(H)).cpu().numpy()
    assert got.shape == (r, c)
    assert rel_l2(got, oracle.pipeline_padded(img, H)) <= tol_fp32(R * C)


def test_paper_application_460x506_disc(gb):
    """The paper's configuration: a 460 x 506 image padded to 512^2, the disc
    filter of radius 340 (Eq. filtro), the result cut back; and its spectrum."""
    img = synth.sky(460, 506, 200, 52)
    H = synth.disc_filter(512, 512, 340.0)
    got = gb.fft2_filter_ifft2_padded(_cuda(img), _cuda(H)).cpu().numpy()
    assert rel_l2(got, oracle.pipeline_padded(img, H)) <= tol_fp32(512 * 512)
    mag = gb.fft2_spectrum(_cuda(img)).cpu().numpy()
    assert mag.shape == (512, 512)
    assert rel_l2(mag, oracle.spectrum_padded(img, 512, 512)) <= tol_fp32(512 * 512)


def test_padded_batch_per_image_filters_in_place(gb):
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    B, r, c, R, C = 4, 90, 120, 128, 128
    img = np.stack([synth.sky(r, c, 20, 53, b) for b in range(B)])
    H = np.stack([synth.gaussian_lowpass(R, C, 3.0 + 4 * b) for b in range(B)])
    plan = gb.Plan2D(R, C, B, "cuda", {nat.OPT_H_BATCH_STRIDE: R * C, nat.OPT_IMAGES_PER_CHUNK: 3})
    t = _cuda(img)
    plan.filter_padded(t, _cuda(H), out=t)
    torch.cuda.synchronize()
    assert max_rel_l2(t.cpu().numpy(), oracle.pipeline_padded(img, H), axes=(1, 2)) <= tol_fp32(R * C)


@pytest.mark.parametrize("r,c,R,C", [(256, 128, 256, 128), (7, 13, 8, 16), (2, 2, 2, 2), (1000, 3, 1024, 4),
                                     (512, 4096, 512, 4096), (30, 8192, 32, 8192)])
def test_spectrum(gb, r, c, R, C):
    img = synth.sky(r, c, max(1, r * c // 3000), 54, r, c)
    got = gb.fft2_spectrum(_cuda(img), R, C).cpu().numpy()
    assert rel_l2(got, oracle.spectrum_padded(img, R, C)) <= tol_fp32(R * C)


def test_spectrum_batch_and_eq5(gb):
    img = np.stack([synth.sky(60, 100, 10, 55, b) for b in range(3)])
    got = gb.fft2_spectrum(_cuda(img), 64, 128).cpu().numpy()
    assert max_rel_l2(got, oracle.spectrum_padded(img, 64, 128), axes=(1, 2)) <= tol_fp32(64 * 128)
    got5 = gb.fft2_spectrum(_cuda(img), 64, 128, eq5=True).cpu().numpy()
    assert max_rel_l2(got5, oracle.spectrum_padded(img, 64, 128, 1), axes=(1, 2)) <= tol_fp32(64 * 128)


def test_spectrum_closed_forms(gb):
    """Delta -> every bin 1/(R C); constant -> only DC; one cosine -> two bins of 1/2."""
    R, C = 64, 32
    d = np.zeros((50, 20), np.float32)
    d[0, 0] = 1
    mag = gb.fft2_spectrum(_cuda(d), R, C).cpu().numpy()
    assert np.max(np.abs(mag - 1.0 / (R * C))) <= 1e-7 / (R * C) * 10
    y, x = np.mgrid[0:R, 0:C]
    cosimg = np.cos(2 * np.pi * (5 * y / R + 3 * x / C)).astype(np.float32)
    mag = gb.fft2_spectrum(_cuda(cosimg)).cpu().numpy()
    want = np.zeros((R, C))
    want[5, 3] = want[R - 5, C - 3] = 0.5
    assert np.max(np.abs(mag - want)) <= 1e-6


def test_spectrum_then_filter_on_one_plan(gb):
    """The spectrum uses the plan's filter workspace as scratch; the next
    filter call prepares its filter again."""
    import torch

    plan = gb.Plan2D(512, 512, 1, "cuda")
    img = synth.sky(512, 512, 30, 56)
    H = synth.gaussian_lowpass(512, 512, 10.0)
    ti, th = _cuda(img), _cuda(H)
    out = plan.filter(ti, th)
    plan.spectrum(ti)
    out2 = plan.filter(ti, th)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
