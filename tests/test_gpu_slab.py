"""GPU parity of the row-slab decomposition (fft2_slab_*): one image split
over R ranks, every rank's kernels run on one device through the sharded
code path (Plan2DSlab, exchanges done as local copies), against the FP64
oracle's pipeline and against the one-rank entry point."""

import ctypes

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import rel_l2, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch

    import paper_cs_0103001_gb300 as gb

    assert torch.cuda.is_available()
    return gb


# (rows, cols, ranks): TMA column pass with 2, 4 and 16 runs per column at 4096
# rows; the one-column-per-block kernel elsewhere; tall, wide and 8 ranks
CASES = [(4096, 4096, 2), (4096, 4096, 4), (4096, 1024, 16), (512, 1024, 4), (1024, 2048, 8), (8192, 512, 2),
         (2048, 32, 4), (512, 64, 2), (256, 256, 2)]


@pytest.mark.parametrize("rows,cols,nranks", CASES)
def test_sharded_matches_oracle(gb, rows, cols, nranks):
    import torch

    img = synth.sky(rows, cols, max(5, rows * cols // 2000), 40, rows, cols)
    H = synth.random_filter(rows, cols, 41, rows, cols)
    ti, th = torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()
    out = gb.fft2_filter_ifft2_sharded(ti, th, nranks=nranks)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.pipeline(img, H)
    tol = tol_fp32(rows * cols)
    err = rel_l2(got, ref)
    assert err <= tol, f"rel-L2 {err:.3e} > {tol:.3e}"
    one = gb.fft2_filter_ifft2(ti, th).cpu().numpy()
    assert rel_l2(got, one) <= tol


def test_rank_writes_only_its_rows(gb):
    import torch

    from paper_cs_0103001_gb300 import slab

    rows, cols, R = 512, 1024, 4
    img = torch.from_numpy(synth.sky(rows, cols, 100, 42)).cuda()
    H = torch.from_numpy(synth.gaussian_lowpass(rows, cols, 40.0)).cuda()
    plans = [gb.Plan2DSlab(rows, cols, R, r, "cuda") for r in range(R)]
    n = plans[0].exchange_elems
    assert n == (cols // 2) * (rows // R)
    sends = torch.empty(R, R, n // R, dtype=torch.complex64, device="cuda")
    for r, p in enumerate(plans):
        p.rows_forward(img, sends[r])
    recvs = sends.transpose(0, 1).contiguous()
    for q, p in enumerate(plans):
        p.columns(recvs[q], H)
    backs = recvs.transpose(0, 1).contiguous()
    out = torch.full_like(img, float("nan"))
    plans[1].rows_inverse(backs[1], out)
    torch.cuda.synchronize()
    written = ~torch.isnan(out).any(dim=1).cpu().numpy()
    assert sorted(np.nonzero(written)[0].tolist()) == sorted(slab.slab_rows(rows, R, 1))
    ref = oracle.pipeline(img.cpu().numpy(), H.cpu().numpy())
    mine = slab.slab_rows(rows, R, 1)
    assert rel_l2(out.cpu().numpy()[mine], ref[mine]) <= tol_fp32(rows * cols)


def test_slab_plan_rejects_bad_decompositions(gb):
    from paper_cs_0103001_gb300 import _native as nat

    h = ctypes.c_void_p()
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 3, 0, ctypes.byref(h)) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_slab_plan_create(128, 128, 2, 0, ctypes.byref(h)) == nat.ERR_INVALID_SIZE
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 2, 2, ctypes.byref(h)) == nat.ERR_INVALID_VALUE
    assert nat.lib.fft2_slab_plan_create(4096, 4096, 2, -1, ctypes.byref(h)) == nat.ERR_INVALID_VALUE
