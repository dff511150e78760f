"""GPU parity of the batched (uneven sizes, per-image filter) pipeline, in
both forms: the one-shape kernels once per shape class (default) and four
persistent launches over largest-first work lists; optionally replayed from a
captured CUDA graph."""

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


SHAPES = [(16, 16), (2048, 2048), (64, 256), (512, 32), (4096, 16), (16, 4096), (128, 128), (1024, 512),
          (256, 2048), (32, 32), (64, 64)]


def _inputs(shapes, tag):
    imgs = [synth.sky(r, c, max(1, r * c // 4000), tag, i) for i, (r, c) in enumerate(shapes)]
    Hs = [synth.random_filter(r, c, tag + 1, i) for i, (r, c) in enumerate(shapes)]
    return imgs, Hs


def test_mixed_shapes_against_oracle(gb):
    import torch

    imgs, Hs = _inputs(SHAPES, 40)
    outs = gb.fft2_filter_ifft2_batched([torch.from_numpy(a).cuda() for a in imgs],
                                        [torch.from_numpy(h).cuda() for h in Hs])
    for (r, c), a, h, o in zip(SHAPES, imgs, Hs, outs):
        assert rel_l2(o.cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(r * c), (r, c)


@pytest.mark.parametrize("form", [0, 1])
def test_both_forms_against_oracle(gb, form):
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    shapes = SHAPES + [(2048, 2048), (64, 256), (16, 16)]  # repeated shapes share a class
    imgs, Hs = _inputs(shapes, 47)
    plan = gb.Plan2DBatched(shapes, "cuda", {nat.OPT_BATCH_FORM: form})
    outs = plan.filter([torch.from_numpy(a).cuda() for a in imgs], [torch.from_numpy(h).cuda() for h in Hs])
    for (r, c), a, h, o in zip(shapes, imgs, Hs, outs):
        assert rel_l2(o.cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(r * c), (form, r, c)
    assert plan.check_guards() == 0


def test_graph_replay_and_plain_launches_agree(gb):
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    imgs, Hs = _inputs(SHAPES, 42)
    ti = [torch.from_numpy(a).cuda() for a in imgs]
    th = [torch.from_numpy(h).cuda() for h in Hs]
    plan = gb.Plan2DBatched(SHAPES, "cuda")
    first = [o.clone() for o in plan.filter(ti, th)]
    second = plan.filter(ti, th)  # replays the captured graph
    for a, b in zip(first, second):
        assert torch.equal(a, b)
    plain = gb.Plan2DBatched(SHAPES, "cuda", {nat.OPT_USE_GRAPH: 0}).filter(ti, th)
    for a, b in zip(first, plain):
        assert torch.equal(a, b)
    # the same images through the one-shape plans give the same numbers
    for (r, c), a, h, o in zip(SHAPES, ti, th, first):
        ref = gb.fft2_filter_ifft2(a, h)
        assert rel_l2(o.cpu().numpy(), ref.cpu().numpy()) <= tol_fp32(r * c)


def test_new_pointers_reach_the_captured_graph(gb):
    import torch

    shapes = [(256, 256), (64, 128)]
    plan = gb.Plan2DBatched(shapes, "cuda")
    for tag in (44, 45):
        imgs, Hs = _inputs(shapes, tag)
        outs = plan.filter([torch.from_numpy(a).cuda() for a in imgs], [torch.from_numpy(h).cuda() for h in Hs])
        for (r, c), a, h, o in zip(shapes, imgs, Hs, outs):
            assert rel_l2(o.cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(r * c)


def test_bind_and_run(gb):
    """run() over bound buffers gives filter()'s numbers; a filter() call
    unbinds, so run() then refuses."""
    import torch

    imgs, Hs = _inputs(SHAPES, 44)
    ti = [torch.from_numpy(a).cuda() for a in imgs]
    th = [torch.from_numpy(h).cuda() for h in Hs]
    plan = gb.Plan2DBatched(SHAPES, "cuda")
    with pytest.raises(RuntimeError):
        plan.run()
    ref = [o.clone() for o in plan.filter(ti, th)]
    outs = [torch.full_like(a, float("nan")) for a in ti]
    plan.bind(ti, th, outs)
    plan.run()
    plan.run()
    for a, b in zip(ref, outs):
        assert torch.equal(a, b)
    plan.filter(ti, th)
    with pytest.raises(RuntimeError):
        plan.run()


def test_autotune_keeps_results(gb):
    import torch

    imgs, Hs = _inputs(SHAPES, 46)
    ti = [torch.from_numpy(a).cuda() for a in imgs]
    th = [torch.from_numpy(h).cuda() for h in Hs]
    plan = gb.Plan2DBatched(SHAPES, "cuda")
    before = [o.clone() for o in plan.filter(ti, th)]
    packed = plan.autotune(ti, th)
    assert all(1 <= (packed >> (8 * s)) & 0xFF <= 64 for s in range(4))
    after = plan.filter(ti, th)
    for (r, c), a, h, b in zip(SHAPES, imgs, Hs, after):  # either form: the oracle's result
        assert rel_l2(b.cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(r * c)


def test_uneven_workload_sampled():
    """512 skies with sides drawn from {64..2048}, each with its own Gaussian
    low-pass (sigma uniform in [8, 128] bins); every 16th image against the
    oracle, all images against the one-shape path."""
    import torch

    import paper_cs_0103001_gb300 as gb

    batch = synth.uneven_batch(512, 4)
    ti = [torch.from_numpy(a).cuda() for a, _, _ in batch]
    th = [torch.from_numpy(h).cuda() for _, h, _ in batch]
    outs = gb.fft2_filter_ifft2_batched(ti, th)
    for i in range(0, 512, 16):
        a, h, _ = batch[i]
        assert rel_l2(outs[i].cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(a.size), i
    for i, (a, h) in enumerate(zip(ti, th)):
        if i % 5 == 0:
            ref = gb.fft2_filter_ifft2(a, h)
            assert rel_l2(outs[i].cpu().numpy(), ref.cpu().numpy()) <= tol_fp32(a.numel())


def test_autotune_first_in_a_fresh_process():
    """Tuning before any other batched call (so no kernel attribute has been
    set yet in the process) must work."""
    import os
    import subprocess
    import sys

    code = (
        "import torch, paper_cs_0103001_gb300 as gb\n"
        "from paper_cs_0103001_gb300 import synth\n"
        "b = synth.uneven_batch(12, 7)\n"
        "ti = [torch.from_numpy(a).cuda() for a, _, _ in b]\n"
        "th = [torch.from_numpy(h).cuda() for _, h, _ in b]\n"
        "p = gb.Plan2DBatched([tuple(a.shape) for a in ti], 'cuda')\n"
        "print(p.autotune(ti, th))\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "PYTHONPATH": root})
    assert r.returncode == 0, r.stderr[-2000:]
