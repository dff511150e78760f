"""GPU parity of the pipeline's adjoint (grad wrt the image and the filter)
against the oracle's closed forms, and against FP64 central finite
differences of the oracle's loss."""

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import max_rel_l2, rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5  # two transforms deep in fp32


@pytest.fixture(scope="module")
def gb():
    import torch

    import paper_cs_0103001_gb300 as gb

    assert torch.cuda.is_available()
    return gb


@pytest.mark.parametrize("rows,cols,batch", [(2, 2, 1), (8, 4, 2), (16, 64, 3), (64, 16, 2), (128, 128, 4),
                                             (256, 512, 2), (1024, 32, 2), (32, 1024, 2)])
def test_backward_matches_oracle(gb, rows, cols, batch):
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    img = np.stack([synth.sky(rows, cols, 5, 30, b) for b in range(batch)])
    H = synth.random_filter(rows, cols, 31, rows)
    G = synth.real_uniform((batch, rows, cols), 32, rows)
    gi_ref, gh_ref = oracle.pipeline_grad(img, H, G)
    for chunk in (0, 1):  # default chunking, and one image per chunk (grad_H accumulated)
        plan = gb.Plan2D(rows, cols, batch, "cuda", {nat.OPT_ENABLE_BACKWARD: 1, nat.OPT_IMAGES_PER_CHUNK: chunk})
        gi = torch.empty(batch, rows, cols, device="cuda")
        gh = torch.empty(rows, cols, device="cuda")
        plan.backward(torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda(), torch.from_numpy(G).cuda(), gi, gh)
        assert max_rel_l2(gi.cpu().numpy(), gi_ref, axes=(1, 2)) <= GRAD_TOL
        assert rel_l2(gh.cpu().numpy(), gh_ref) <= GRAD_TOL


def test_autograd_mse_against_finite_differences(gb):
    """loss = mean((pipeline(noisy, H) - clean)^2); 32 entries of each
    gradient against FP64 central differences of the oracle's loss (the loss
    is quadratic in img for fixed H and in H for fixed img, so the central
    difference has no truncation error)."""
    import torch

    rows, cols, batch = 64, 128, 3
    clean = np.stack([synth.sky(rows, cols, 8, 33, b) for b in range(batch)])
    noisy = (clean + synth.real_uniform(clean.shape, 34, low=-20, high=20)).astype(np.float32)
    H0 = (1.0 + 0.1 * synth.real_uniform((rows, cols), 35)).astype(np.float32)
    x = torch.from_numpy(noisy).cuda().requires_grad_(True)
    Ht = torch.from_numpy(H0).cuda().requires_grad_(True)
    c = torch.from_numpy(clean).cuda()
    loss = torch.mean((gb.fft2_filter_ifft2(x, Ht) - c) ** 2)
    loss.backward()
    gx, gH = x.grad.cpu().numpy(), Ht.grad.cpu().numpy()

    def L(im, h):
        return float(np.mean((oracle.pipeline(im, h) - clean) ** 2))

    g = np.random.default_rng(36)
    base_img = noisy.astype(np.float64)
    base_H = H0.astype(np.float64)
    for _ in range(32):
        b, r, q = g.integers(batch), g.integers(rows), g.integers(cols)
        e = np.zeros_like(base_img)
        e[b, r, q] = 1.0
        fd = (L(base_img + e, base_H) - L(base_img - e, base_H)) / 2.0
        assert abs(gx[b, r, q] - fd) <= 1e-5 * max(abs(fd), np.max(np.abs(gx)))
        e = np.zeros_like(base_H)
        e[r, q] = 1e-2
        fd = (L(base_img, base_H + e) - L(base_img, base_H - e)) / 2e-2
        assert abs(gH[r, q] - fd) <= 1e-5 * max(abs(fd), np.max(np.abs(gH)))


def test_backward_differentiable_workload_size(gb):
    """16 x 2048^2 noisy skies, H = 1: full gradients against the oracle."""
    import torch

    rows = cols = 2048
    batch = 16
    clean = np.stack([synth.sky(rows, cols, 5000, 5, b) for b in range(batch)])
    noisy = (clean + synth.real_uniform(clean.shape, 5, 99, low=-30, high=30)).astype(np.float32)
    H = np.ones((rows, cols), np.float32)
    x = torch.from_numpy(noisy).cuda().requires_grad_(True)
    Ht = torch.from_numpy(H).cuda().requires_grad_(True)
    loss = torch.mean((gb.fft2_filter_ifft2(x, Ht) - torch.from_numpy(clean).cuda()) ** 2)
    loss.backward()
    y = oracle.pipeline(noisy, H)
    G = 2.0 * (y - clean) / y.size
    gi_ref, gh_ref = oracle.pipeline_grad(noisy, H, G)
    assert max_rel_l2(x.grad.cpu().numpy(), gi_ref, axes=(1, 2)) <= GRAD_TOL
    gh = Ht.grad.cpu().numpy().astype(np.float64)
    # grad_H = s sum_b Re(conj(W G_b) W x_b) multiplies two fp32 spectra whose
    # errors are bounded normwise by the transform tolerance g = 2e-7 log2(NM)
    # (||dW x|| <= g ||W x||).  Hence ||d grad_H|| <= 2 g s sum_b ||W G_b|| ||W x_b||
    # = 2 g sum_b ||G_b|| ||x_b|| (Parseval, s = 1/(NM)).  The relative form of
    # this bound is large here because the sky's background (100 per pixel)
    # dominates ||x|| while grad_H lives at the frequencies of the noise.
    g = 2e-7 * np.log2(rows * cols)
    bound = 2 * g * sum(np.linalg.norm(G[b]) * np.linalg.norm(noisy[b].astype(np.float64)) for b in range(batch))
    assert np.linalg.norm(gh - gh_ref) <= bound
