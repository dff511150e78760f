"""GPU parity of the Sec. 5 pipeline out = Re(ifft2(H . fft2(img))) against
the FP64 oracle, on the same float32 inputs, through the C ABI."""

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


def _pipe(gb, img, H):
    import torch

    out = gb.fft2_filter_ifft2(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda())
    return out.cpu().numpy()


SHAPES = [(2, 2), (2, 16), (16, 2), (4, 8), (8, 8), (16, 32), (32, 16), (64, 64), (128, 256), (256, 128),
          (512, 512), (1024, 64), (64, 1024), (2048, 256), (256, 2048), (4096, 32), (32, 4096), (8192, 16),
          (16, 8192)]


@pytest.mark.parametrize("rows,cols", SHAPES)
def test_shapes_random_filter(gb, rows, cols):
    """Every row/column length, with a filter that has no symmetry at all."""
    img = synth.sky(rows, cols, max(1, rows * cols // 2000), 10, rows, cols)
    H = synth.random_filter(rows, cols, 11, rows, cols)
    assert rel_l2(_pipe(gb, img, H), oracle.pipeline(img, H)) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("rows,cols", [(256, 256), (512, 1024), (2048, 2048)])
def test_smooth_filters(gb, rows, cols):
    img = synth.sky(rows, cols, 50, 12, rows)
    for H in (synth.gaussian_lowpass(rows, cols, 16.0), synth.butterworth_lowpass(rows, cols, 4, 0.1),
              synth.disc_filter(rows, cols, rows * 340 / 512)):
        assert rel_l2(_pipe(gb, img, H), oracle.pipeline(img, H)) <= tol_fp32(rows * cols)


def test_identity_and_mean(gb):
    img = synth.sky(128, 64, 20, 13)
    out = _pipe(gb, img, np.ones((128, 64), np.float32))
    assert rel_l2(out, img.astype(np.float64)) <= tol_fp32(128 * 64)
    d = np.zeros((128, 64), np.float32)
    d[0, 0] = 1
    out = _pipe(gb, img, d)
    assert np.max(np.abs(out - img.astype(np.float64).mean())) <= 1e-5 * abs(img.mean())


def test_batch_per_image_filter_and_chunks(gb):
    """Batch of 5 images, each with its own filter, processed one image per
    workspace chunk, in place (img == out)."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    rows, cols, B = 256, 512, 5
    img = np.stack([synth.sky(rows, cols, 40, 14, b) for b in range(B)])
    H = np.stack([synth.gaussian_lowpass(rows, cols, 4.0 + 10 * b) for b in range(B)])
    ref = oracle.pipeline(img, H)
    plan = gb.Plan2D(rows, cols, B, "cuda", {nat.OPT_H_BATCH_STRIDE: rows * cols, nat.OPT_IMAGES_PER_CHUNK: 1})
    t = torch.from_numpy(img).cuda()
    plan.filter(t, torch.from_numpy(H).cuda(), out=t)
    assert max_rel_l2(t.cpu().numpy(), ref, axes=(1, 2)) <= tol_fp32(rows * cols)
    # shared filter through the autograd front end, batch dims flattened
    out = gb.fft2_filter_ifft2(torch.from_numpy(img).cuda().reshape(B, 1, rows, cols),
                               torch.from_numpy(H[2]).cuda()).cpu().numpy()
    assert max_rel_l2(out.reshape(B, rows, cols), oracle.pipeline(img, H[2]), axes=(1, 2)) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("rows,cols,chunk", [(4096, 64, 3), (4096, 16, 0), (4096, 512, 2), (2048, 256, 2),
                                             (2048, 4, 0), (1024, 128, 0), (1024, 8, 3)])
def test_tall_batches_through_the_persistent_column_pass(gb, rows, cols, chunk):
    """Batches of tall images, several per launch, with per-image filters and
    row-pass groups from 2 to 256 pairs: 4096 rows take the persistent
    TMA-fed column pass (columns of consecutive images in one walk), 1024 and
    2048 rows the kernel with several columns per block."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    B = 3
    img = np.stack([synth.sky(rows, cols, 60, 16, b) for b in range(B)])
    H = np.stack([synth.random_filter(rows, cols, 17, b) for b in range(B)])
    plan = gb.Plan2D(rows, cols, B, "cuda", {nat.OPT_H_BATCH_STRIDE: rows * cols, nat.OPT_IMAGES_PER_CHUNK: chunk,
                                            nat.OPT_PROFILE: 1})
    got = plan.filter(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()).cpu().numpy()
    plan.device_status()
    assert max_rel_l2(got, oracle.pipeline(img, H), axes=(1, 2)) <= tol_fp32(rows * cols)


def test_repeatable_bits(gb):
    import torch

    img = torch.from_numpy(synth.sky(1024, 1024, 100, 15)).cuda()
    H = torch.from_numpy(synth.gaussian_lowpass(1024, 1024, 30.0)).cuda()
    a = gb.fft2_filter_ifft2(img, H)
    b = gb.fft2_filter_ifft2(img, H)
    assert torch.equal(a, b)


@pytest.mark.parametrize("cfg", ["256_gauss32", "4096_butterworth"])
def test_workload_sizes(gb, cfg):
    """The two single-image workloads at full size: 256^2 sky (50 sources,
    Gaussian sigma 32 bins) and 4096^2 sky (20000 sources, Butterworth order 4,
    cutoff 0.1 Nyquist); whole output image against the oracle."""
    if cfg == "256_gauss32":
        img = synth.sky(256, 256, 50, 1)
        H = synth.gaussian_lowpass(256, 256, 32.0)
    else:
        img = synth.sky(4096, 4096, 20000, 3)
        H = synth.butterworth_lowpass(4096, 4096, 4, 0.1)
    n = img.size
    got = _pipe(gb, img, H)
    ref = oracle.pipeline(img, H)
    assert rel_l2(got, ref) <= tol_fp32(n)
    # sampled pixels straight from the spectrum (Eq. E3 summed directly)
    if n <= 1 << 16:
        F = oracle.fft2(img) * H
        rows, cols = img.shape
        for (x, y) in ((0, 0), (17, 200), (255, 3)):
            px = np.sum(F * np.exp(2j * np.pi * (np.arange(rows)[:, None] * x / rows
                                                 + np.arange(cols)[None, :] * y / cols))).real
            assert abs(got[x, y] - px) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("rows,cols,batch", [(4096, 64, 3), (4096, 1024, 1)])
def test_column_pass_forms(gb, form, rows, cols, batch):
    """Each form of the column pass over 4096-row columns (GBFFT_OPT_COLUMN_FORM:
    TMA-fed with the filter in shared or global memory, one column per block)
    against the oracle, with per-image filters over several images."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    img = np.stack([synth.sky(rows, cols, 60, 15, b) for b in range(batch)])
    H = np.stack([synth.random_filter(rows, cols, 16, b) for b in range(batch)])
    plan = gb.Plan2D(rows, cols, batch, "cuda", {nat.OPT_H_BATCH_STRIDE: rows * cols, nat.OPT_COLUMN_FORM: form})
    out = plan.filter(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()).cpu().numpy()
    assert max_rel_l2(out, oracle.pipeline(img, H), axes=(1, 2)) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("per_image,chunk", [(True, 1), (True, 0), (False, 1), (False, 0)])
def test_4096_filters_per_image_and_shared_over_chunks(gb, per_image, chunk):
    """4096^2 images with asymmetric filters (the mirror terms of the
    prepared filter matter): per-image filters, or one filter shared by every
    image (prepared once per call, by the first chunk), one or all images per
    chunk.  Column forms 1 and 2 read the same prepared filter from shared or
    global memory with the same arithmetic, so they agree bit for bit; both
    match the oracle."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    rows = cols = 4096
    B = 3 if per_image else 2
    img = np.stack([synth.sky(rows, cols, 3000, 18, b) for b in range(B)])
    H = (np.stack([synth.random_filter(rows, cols, 19, b) for b in range(B)]) if per_image
         else synth.random_filter(rows, cols, 19, 7))
    opts = {nat.OPT_H_BATCH_STRIDE: rows * cols if per_image else 0, nat.OPT_IMAGES_PER_CHUNK: chunk}
    ti, th = torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()
    smem = gb.Plan2D(rows, cols, B, "cuda", {**opts, nat.OPT_COLUMN_FORM: 1}).filter(ti, th)
    glob = gb.Plan2D(rows, cols, B, "cuda", {**opts, nat.OPT_COLUMN_FORM: 2}).filter(ti, th)
    assert torch.equal(smem, glob)
    ref = oracle.pipeline(img, H)
    assert max_rel_l2(smem.cpu().numpy(), ref, axes=(1, 2)) <= tol_fp32(rows * cols)


@pytest.mark.parametrize("rows,cols,batch,chunk", [(4096, 4096, 2, 0), (1024, 512, 5, 2), (256, 256, 3, 0)])
def test_prepared_filter(gb, rows, cols, batch, chunk):
    """One filter prepared once and used by later calls: equal to the plain
    pipeline with that filter (bit for bit where both take the same kernels,
    within the tolerance at 256^2, where the plain call takes the on-chip
    path) and to the oracle; calls that reuse the workspace discard it."""
    import ctypes

    import torch

    from paper_cs_0103001_gb300 import _native as nat

    img = np.stack([synth.sky(rows, cols, 200, 20, b) for b in range(batch)])
    H = synth.random_filter(rows, cols, 21)
    H2 = synth.gaussian_lowpass(rows, cols, 30.0)
    ti, th, th2 = torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda(), torch.from_numpy(H2).cuda()
    plan = gb.Plan2D(rows, cols, batch, "cuda", {nat.OPT_IMAGES_PER_CHUNK: chunk})
    plan.prepare_filter(th)
    a = plan.filter_prepared(ti)
    b = plan.filter_prepared(ti)  # the prepared filter stays
    assert torch.equal(a, b)
    ref = oracle.pipeline(img, H)
    assert max_rel_l2(a.cpu().numpy(), ref, axes=(1, 2)) <= tol_fp32(rows * cols)
    plain = plan.filter(ti, th)  # discards the prepared filter
    if rows > 256:
        assert torch.equal(a, plain)
    with pytest.raises(nat.GbfftError):
        plan.filter_prepared(ti)
    plan.prepare_filter(th2)
    c = plan.filter_prepared(ti)
    assert max_rel_l2(c.cpu().numpy(), oracle.pipeline(img, H2), axes=(1, 2)) <= tol_fp32(rows * cols)
    # per-image filters: not this call's business
    per = gb.Plan2D(rows, cols, batch, "cuda", {nat.OPT_H_BATCH_STRIDE: rows * cols})
    assert nat.lib.fft2_filter_prepare(per.handle, ctypes.c_void_p(th.data_ptr()), None) == nat.ERR_UNSUPPORTED


def test_largest_image_8192_squared(gb):
    """The largest 2D plan, 8192 x 8192 (rows of 8192: 1024-thread row
    blocks; columns of 8192: one column per block), with an asymmetric
    filter, against the oracle."""
    rows = cols = 8192
    img = synth.sky(rows, cols, 20000, 22)
    H = synth.random_filter(rows, cols, 23)
    assert rel_l2(_pipe(gb, img, H), oracle.pipeline(img, H)) <= tol_fp32(rows * cols)
