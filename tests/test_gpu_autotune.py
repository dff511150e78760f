"""The autotuner (fft_plan_autotune): every candidate it may choose gives the
oracle's result, its choice lands in the JSON cache keyed by GPU and shape,
a cached choice is applied without timing, and an unreadable cache only
means tuning again."""

import json

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


def _device_key():
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def _pipeline_case(rows, cols, batch, seed):
    img = np.stack([synth.sky(rows, cols, 40, seed, b) for b in range(batch)])
    H = np.stack([synth.random_filter(rows, cols, seed + 1, b) for b in range(batch)])
    return img, H


def test_autotune_2d_choice_is_cached_and_reused(gb, tmp_path, monkeypatch):
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    path = tmp_path / "tune.json"
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(path))
    rows, cols, batch = 4096, 64, 2
    img, H = _pipeline_case(rows, cols, batch, 50)
    ti, th = torch.from_numpy(img).cuda(), torch.from_numpy(H).cuda()
    opts = {nat.OPT_H_BATCH_STRIDE: rows * cols}
    plan = gb.Plan2D(rows, cols, batch, "cuda", opts)
    chosen = plan.autotune(ti, th)
    assert chosen["column_form"] in (1, 2, 3)
    ref = oracle.pipeline(img, H)
    assert max_rel_l2(plan.filter(ti, th).cpu().numpy(), ref, axes=(1, 2)) <= tol_fp32(rows * cols)
    data = json.loads(path.read_text())
    key = f"{_device_key()}|2d:r=12:c=6:b=2:h=1:p=0:bw=0"
    assert data["entries"][key]["column_form"] == chosen["column_form"]
    assert data["entries"][key]["us"] > 0
    # a stored choice is applied as it stands (here edited to the one-column form)
    data["entries"][key]["column_form"] = 3
    path.write_text(json.dumps(data))
    plan2 = gb.Plan2D(rows, cols, batch, "cuda", opts)
    assert plan2.autotune(ti, th)["column_form"] == 3
    assert max_rel_l2(plan2.filter(ti, th).cpu().numpy(), ref, axes=(1, 2)) <= tol_fp32(rows * cols)


def test_autotune_small_2d_and_unreadable_cache(gb, tmp_path, monkeypatch):
    import torch

    path = tmp_path / "tune.json"
    path.write_text("{this is not json")
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(path))
    rows = cols = 256
    img, H = _pipeline_case(rows, cols, 1, 52)
    ti, th = torch.from_numpy(img[0]).cuda(), torch.from_numpy(H[0]).cuda()
    plan = gb.Plan2D(rows, cols, 1, "cuda")
    chosen = plan.autotune(ti, th)
    assert chosen["onchip"] in (0, 1)
    assert rel_l2(plan.filter(ti, th).cpu().numpy(), oracle.pipeline(img[0], H[0])) <= tol_fp32(rows * cols)
    assert "entries" in json.loads(path.read_text())  # rewritten as valid JSON
    # no cache at all: tuning still works
    monkeypatch.setenv("GBFFT_TUNE_CACHE", "")
    assert gb.Plan2D(rows, cols, 1, "cuda").autotune(ti, th)["onchip"] in (0, 1)


def test_autotune_1d_cluster_or_four_step(gb, tmp_path, monkeypatch):
    import torch

    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(tmp_path / "tune.json"))
    n, batch = 1 << 16, 4
    x = synth.complex_uniform((batch, n), 53)
    tx = torch.from_numpy(x).cuda()
    plan = gb.Plan1D(n, batch, torch.complex64, "cuda")
    assert plan.autotune(tx) in (1, 2)
    got = plan.forward(tx).cpu().numpy()
    assert max_rel_l2(got, oracle.fft(x), axes=(1,)) <= tol_fp32(n)
