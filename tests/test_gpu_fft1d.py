"""GPU parity of the batched 1D transforms (Eq. E2 forward, Eq. E3 inverse)
against the FP64 oracle, through the C ABI (via the ctypes binding)."""

import numpy as np
import pytest

import oracle
from paper_cs_0103001_gb300 import synth
from tests.gpu_util import FP64_TOL, max_rel_l2, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch

    import paper_cs_0103001_gb300 as gb

    assert torch.cuda.is_available()
    return gb


def _run(gb, x, inverse=False, dtype=None):
    import torch

    t = torch.from_numpy(x).cuda()
    if dtype is not None:
        t = t.to(dtype)
    y = gb.ifft(t) if inverse else gb.fft(t)
    return y.cpu().numpy()


def _tol(n, dbl):
    return FP64_TOL if dbl else tol_fp32(n)


@pytest.mark.parametrize("dbl", [False, True], ids=["c64", "c128"])
@pytest.mark.parametrize("log2n", range(1, 15))
@pytest.mark.parametrize("batch", [1, 3, 17])
def test_one_pass_all_sizes(gb, log2n, batch, dbl):
    import torch

    if dbl and log2n > 13:
        pytest.skip("complex128 one-pass limit is 2^13 (four-step beyond)")
    n = 1 << log2n
    x = synth.complex_uniform((batch, n), 2, log2n, batch)
    dt = torch.complex128 if dbl else None
    xo = x.astype(np.complex128)
    got = _run(gb, x, dtype=dt)
    assert max_rel_l2(got, oracle.fft(xo), axes=-1) <= _tol(n, dbl)
    got = _run(gb, x, inverse=True, dtype=dt)
    assert max_rel_l2(got, oracle.ifft(xo), axes=-1) <= _tol(n, dbl)


@pytest.mark.parametrize("dbl,log2n,batch", [
    (False, 15, 3), (False, 16, 2), (False, 17, 3), (False, 18, 1), (False, 20, 2), (False, 21, 1), (False, 22, 1),
    (False, 23, 1), (False, 24, 1),
    (True, 14, 3), (True, 15, 2), (True, 17, 1), (True, 19, 2),
])
def test_four_step(gb, dbl, log2n, batch):
    import torch

    n = 1 << log2n
    x = synth.complex_uniform((batch, n), 2, log2n, batch)
    dt = torch.complex128 if dbl else None
    xo = x.astype(np.complex128)
    assert max_rel_l2(_run(gb, x, dtype=dt), oracle.fft(xo), axes=-1) <= _tol(n, dbl)
    assert max_rel_l2(_run(gb, x, inverse=True, dtype=dt), oracle.ifft(xo), axes=-1) <= _tol(n, dbl)


def test_in_place_and_plan_reuse(gb):
    import torch

    for n, batch in ((4096, 5), (1 << 16, 3)):
        x = synth.complex_uniform((batch, n), 3, n)
        plan = gb.Plan1D(n, batch, torch.complex64, "cuda")
        t = torch.from_numpy(x).cuda()
        plan.forward(t, out=t)  # in place
        ref = oracle.fft(x.astype(np.complex128))
        assert max_rel_l2(t.cpu().numpy(), ref, axes=-1) <= tol_fp32(n)
        plan.inverse(t, out=t)
        assert max_rel_l2(t.cpu().numpy(), oracle.ifft(ref), axes=-1) <= tol_fp32(n)
        # a second call on the same plan gives the same bits
        a = plan.forward(torch.from_numpy(x).cuda())
        b = plan.forward(torch.from_numpy(x).cuda())
        assert torch.equal(a, b)


def test_closed_forms_on_gpu(gb):
    """delta -> 1/N everywhere; a pure exponential -> one bin."""
    n = 4096
    d = np.zeros((1, n), np.complex64)
    d[0, 0] = 1
    got = _run(gb, d)
    assert np.max(np.abs(got - 1.0 / n)) <= 1e-7 / n * 10
    j = np.arange(n)
    e = np.exp(2j * np.pi * 37 * j / n).astype(np.complex64)[None]
    got = _run(gb, e)[0]
    want = np.zeros(n)
    want[37] = 1
    assert np.max(np.abs(got - want)) < 1e-6


@pytest.mark.parametrize("log2n", [8, 12, 14, 16, 20, 24])
def test_full_size_sweep_sampled(gb, log2n):
    """The 1D sweep configuration: batch * N = 2^26 complex64.  Sampled whole
    transforms against the oracle; every transform checked by the round trip
    inverse(forward(x)) = x."""
    import torch

    n = 1 << log2n
    batch = (1 << 26) // n
    x = synth.complex_uniform((batch, n), 2, log2n)
    t = torch.from_numpy(x).cuda()
    c = gb.fft(t)
    picks = sorted({0, batch - 1, batch // 2, (7 * batch) // 11})[: (2 if log2n >= 22 else 4)]
    ref = oracle.fft(x[picks].astype(np.complex128))
    assert max_rel_l2(c[picks].cpu().numpy(), ref, axes=-1) <= tol_fp32(n)
    f = gb.ifft(c)
    err = torch.sqrt(torch.sum(torch.abs(f - t) ** 2, dim=-1) / torch.sum(torch.abs(t) ** 2, dim=-1))
    assert float(err.max()) <= 2 * tol_fp32(n)


def test_fp64_full_size_sampled(gb):
    """FP64 variant of the sweep: N = 2^20, batch 64."""
    import torch

    n, batch = 1 << 20, 64
    x = synth.complex_uniform((batch, n), 2, 20, 64)
    t = torch.from_numpy(x).cuda().to(torch.complex128)
    c = gb.fft(t)
    picks = [0, 33, 63]
    ref = oracle.fft(x[picks].astype(np.complex128))
    assert max_rel_l2(c[picks].cpu().numpy(), ref, axes=-1) <= FP64_TOL
    bins = np.array([0, 1, 12345, n // 2, n - 1])
    direct = oracle.dft_bins(x[5].astype(np.complex128), bins)
    assert np.max(np.abs(c[5].cpu().numpy()[bins] - direct)) <= 1e-12 * np.sqrt(n) * np.max(np.abs(direct))


@pytest.mark.parametrize("log2n,batch", [(15, 3), (16, 2), (17, 5)])
def test_cluster_path_against_oracle_and_four_step(gb, log2n, batch):
    """With GBFFT_OPT_ONCHIP = 2, lengths 2^15..2^17 run in one thread-block
    cluster per transform (the four-step intermediate in distributed shared
    memory); the launch list shows that kernel; the default (four-step)
    agrees; in place works."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    n = 1 << log2n
    x = synth.complex_uniform((batch, n), 3, log2n, batch)
    xo = x.astype(np.complex128)
    outs = {}
    for onchip in (2, 1):
        plan = gb.Plan1D(n, batch, torch.complex64, "cuda", {nat.OPT_ONCHIP: onchip, nat.OPT_PROFILE: 1})
        t = torch.from_numpy(x).cuda()
        f = plan.forward(t).cpu().numpy()
        b = plan.inverse(t).cpu().numpy()
        plan.forward(t, out=t)  # in place
        torch.cuda.synchronize()
        prof = plan.profile_read()
        assert ("fft1d_cluster" in prof) == (onchip == 2) and ("fourstep_a" in prof) == (onchip != 2)
        assert max_rel_l2(f, oracle.fft(xo), axes=-1) <= tol_fp32(n)
        assert max_rel_l2(b, oracle.ifft(xo), axes=-1) <= tol_fp32(n)
        assert np.array_equal(t.cpu().numpy(), f)
        outs[onchip] = f
    assert max_rel_l2(outs[2], outs[1], axes=-1) <= 2 * tol_fp32(n)


@pytest.mark.parametrize("log2n,batch", [(18, 3), (20, 2), (22, 1), (24, 1)])
def test_tma_four_step_and_device_status(gb, log2n, batch):
    """Complex64 four-step lengths move their tiles with the TMA (pass A: tensor
    loads; pass B: bulk loads and tensor stores); results match the oracle and
    the plan's device status word stays clear."""
    import torch

    n = 1 << log2n
    x = synth.complex_uniform((batch, n), 4, log2n, batch)
    xo = x.astype(np.complex128)
    plan = gb.Plan1D(n, batch, torch.complex64, "cuda")
    t = torch.from_numpy(x).cuda()
    f = plan.forward(t).cpu().numpy()
    b = plan.inverse(t).cpu().numpy()
    plan.device_status()  # raises on a timed-out wait
    assert max_rel_l2(f, oracle.fft(xo), axes=-1) <= tol_fp32(n)
    assert max_rel_l2(b, oracle.ifft(xo), axes=-1) <= tol_fp32(n)


def test_bounded_wait_timeout_is_reported_and_the_plan_stays_usable(gb):
    """The diagnostic block arms an mbarrier that no copy completes: its
    bounded wait runs out, the status word records it, device_status raises
    GBFFT_ERR_TIMEOUT once (and clears it), and the plan's next transform is
    still correct: the context was not lost."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    n, batch = 1 << 20, 1
    plan = gb.Plan1D(n, batch, torch.complex64, "cuda")
    plan.device_status()  # clear
    plan.selftest_wait_timeout(1 << 12)
    with pytest.raises(nat.GbfftError) as err:
        plan.device_status()
    assert err.value.status == nat.ERR_TIMEOUT
    plan.device_status()  # cleared by the read
    x = synth.complex_uniform((batch, n), 6, 20)
    f = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.device_status()
    assert max_rel_l2(f, oracle.fft(x.astype(np.complex128)), axes=-1) <= tol_fp32(n)
    with pytest.raises(nat.GbfftError) as err:
        plan.selftest_wait_timeout(0)  # out of range
    assert err.value.status == nat.ERR_INVALID_VALUE


@pytest.mark.parametrize("passes", [2, 3])
def test_two_and_three_pass_schedules_at_2_24(gb, passes):
    """Length 2^24 (complex64) as two passes of 4096 or three passes of 256
    (GBFFT_OPT_FOURSTEP_PASSES), forward and inverse against the oracle, with
    batch 2 and one transform per workspace chunk (so the chunk loop runs)."""
    import torch

    from paper_cs_0103001_gb300 import _native as nat

    n, batch = 1 << 24, 2
    x = synth.complex_uniform((batch, n), 2, 24, passes)
    plan = gb.Plan1D(n, batch, torch.complex64, "cuda", {nat.OPT_FOURSTEP_PASSES: passes,
                                                         nat.OPT_IMAGES_PER_CHUNK: 1})
    assert plan.get_option(nat.OPT_FOURSTEP_PASSES) == passes
    t = torch.from_numpy(x).cuda()
    xo = x.astype(np.complex128)
    assert max_rel_l2(plan.forward(t).cpu().numpy(), oracle.fft(xo), axes=-1) <= _tol(n, False)
    assert max_rel_l2(plan.inverse(t).cpu().numpy(), oracle.ifft(xo), axes=-1) <= _tol(n, False)
    plan.device_status()
