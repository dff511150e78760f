"""Stand-ins for a memory checker (compute-sanitizer is not available): the
workspace guard bands stay intact after every path of the library, and the
GBFFT_CHECKED build (index-bound checks in the kernels, recording the first
failing site instead of trapping) runs the same paths with no failure and
the oracle's results."""

import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import max_rel_l2, rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Every path of the library, each checked against the oracle; returns the
# plans so that their guard bands can be inspected.  Run here (normal build)
# and in a child process with GBFFT_CHECKED=1.
EXERCISE = r'''
import numpy as np, torch
import oracle
import paper_cs_0103001_gb300 as gb
from paper_cs_0103001_gb300 import _native as nat, synth
from tests.gpu_util import max_rel_l2, rel_l2, tol_fp32

def exercise():
    plans = []
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # 2D pipeline: the TMA-fed shapes, a tall one, the on-chip path, per-image filters
    for rows, cols, batch, per in ((4096, 4096, 1, False), (8192, 512, 1, False), (256, 256, 2, True),
                                   (512, 1024, 3, True), (4096, 64, 2, True)):
        img = np.stack([synth.sky(rows, cols, 30, 60, b) for b in range(batch)])
        H = np.stack([synth.random_filter(rows, cols, 61, b) for b in range(batch)]) if per else synth.random_filter(rows, cols, 61)
        opts = {nat.OPT_H_BATCH_STRIDE: rows * cols} if per else {}
        for form in ((1, 2, 3) if rows == 4096 else (0,)):
            p = gb.Plan2D(rows, cols, batch, "cuda", {**opts, nat.OPT_COLUMN_FORM: form})
            out = p.filter(t(img), t(H)).cpu().numpy()
            assert max_rel_l2(out, oracle.pipeline(img, H), axes=(1, 2)) <= tol_fp32(rows * cols), (rows, cols, form)
            plans.append(p)
    # tensor-core forms
    img = synth.sky(1024, 512, 40, 62)
    H = synth.butterworth_lowpass(1024, 512, 4, 0.1)
    for prec in (1, 2, 3, 4, 5):
        p = gb.Plan2D(1024, 512, 1, "cuda", {nat.OPT_PRECISION: prec})
        out = p.filter(t(img), t(H)).cpu().numpy()
        assert rel_l2(out, oracle.pipeline(img, H)) <= (1 if prec in (2, 4, 5) else 50) * tol_fp32(1024 * 512), prec
        plans.append(p)
    # adjoint, padded, spectrum, analytic
    img = np.stack([synth.sky(256, 512, 30, 63, b) for b in range(2)])
    H = synth.random_filter(256, 512, 64)
    G = synth.real_uniform((2, 256, 512), 65)
    p = gb.Plan2D(256, 512, 2, "cuda", {nat.OPT_ENABLE_BACKWARD: 1})
    gi, gh = torch.empty(2, 256, 512, device="cuda"), torch.empty(256, 512, device="cuda")
    p.backward(t(img), t(H), t(G), gi, gh)
    gi_ref, gh_ref = oracle.pipeline_grad(img, H, G)
    assert max_rel_l2(gi.cpu().numpy(), gi_ref, axes=(1, 2)) <= 1e-5 and rel_l2(gh.cpu().numpy(), gh_ref) <= 1e-5
    plans.append(p)
    p = gb.Plan2D(512, 512, 1, "cuda")
    small = synth.sky(460, 506, 50, 66)
    disc = synth.disc_filter(512, 512, 340.0)
    out = p.filter_padded(t(small), t(disc)).cpu().numpy()
    assert rel_l2(out, oracle.pipeline_padded(small, disc)) <= tol_fp32(512 * 512)
    mag = p.spectrum(t(small)).cpu().numpy()
    assert rel_l2(mag, oracle.spectrum_padded(small, 512, 512)) <= tol_fp32(512 * 512)
    out = p.filter_analytic(t(synth.sky(512, 512, 50, 67)), nat.FILTER_GAUSSIAN, 20.0)
    plans.append(p)
    # the prepared filter
    img = np.stack([synth.sky(1024, 512, 40, 69, b) for b in range(2)])
    H = synth.random_filter(1024, 512, 70)
    p = gb.Plan2D(1024, 512, 2, "cuda")
    p.prepare_filter(t(H))
    out = p.filter_prepared(t(img)).cpu().numpy()
    assert max_rel_l2(out, oracle.pipeline(img, H), axes=(1, 2)) <= tol_fp32(1024 * 512)
    plans.append(p)
    # 1D: one-pass, four-step, cluster, three passes of 256 (2^24)
    for n, batch, onchip in ((4096, 8, 1), (1 << 20, 2, 1), (1 << 16, 4, 2), (1 << 24, 1, 1)):
        x = synth.complex_uniform((batch, n), 68, n)
        p = gb.Plan1D(n, batch, torch.complex64, "cuda", {nat.OPT_ONCHIP: onchip})
        y = p.forward(t(x)).cpu().numpy()
        assert max_rel_l2(y, oracle.fft(x), axes=(1,)) <= tol_fp32(n)
        plans.append(p)
    # batched uneven sizes
    batch = synth.uneven_batch(12, 69)
    ti = [t(a) for a, _, _ in batch]
    th = [t(h) for _, h, _ in batch]
    p = gb.Plan2DBatched([tuple(a.shape) for a in ti], "cuda")
    outs = p.filter(ti, th)
    for (a, h, _), o in zip(batch, outs):
        assert rel_l2(o.cpu().numpy(), oracle.pipeline(a, h)) <= tol_fp32(a.size)
    plans.append(p)
    # one image over 4 emulated ranks (the TMA column pass in runs)
    img = synth.sky(4096, 1024, 100, 70)
    H = synth.random_filter(4096, 1024, 71)
    out = gb.fft2_filter_ifft2_sharded(t(img), t(H), nranks=4).cpu().numpy()
    assert rel_l2(out, oracle.pipeline(img, H)) <= tol_fp32(4096 * 1024)
    torch.cuda.synchronize()
    return plans
'''


def test_guard_bands_intact_after_every_path():
    import ctypes

    import paper_cs_0103001_gb300 as gb  # noqa: F401
    from paper_cs_0103001_gb300 import _native as nat

    ns = {}
    exec(EXERCISE, ns)
    plans = ns["exercise"]()
    assert all(p.check_guards() == 0 for p in plans)
    # the normal build has no index checks
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert nat.lib.gbfft_checked_take(ctypes.byref(a), ctypes.byref(b)) == nat.ERR_UNSUPPORTED


def test_checked_build_runs_every_path_clean():
    import __graft_entry__

    __graft_entry__._build_module().build(checked=True)
    script = EXERCISE + r'''
import ctypes
assert nat.CHECKED and nat.LIB_PATH.endswith("libgbfft_checked.so")
plans = exercise()
assert all(p.check_guards() == 0 for p in plans)
site, fails = ctypes.c_int64(), ctypes.c_int64()
assert nat.lib.gbfft_checked_take(ctypes.byref(site), ctypes.byref(fails)) == nat.OK
print("checked build:", len(plans), "plans, first failing site", site.value, "failures", fails.value)
assert fails.value == 0 and site.value == 0
'''
    env = dict(os.environ, GBFFT_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
