"""Checks that pin the FP64 oracle to facts outside itself.

Each ``pin_*`` function takes an oracle-like object (the ``oracle`` package,
or a deliberately broken copy of it in the mutation tests) and raises
AssertionError when the oracle disagrees with what the paper or the
mathematics fixes: printed values, closed forms, invariants, brute force on
tiny inputs, and numpy's pocketfft (which computes Eq. E2 exactly when asked
for ``norm="forward"``).  None of them re-types the oracle's own formula.
"""

from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

TOL = 1e-12  # FP64: every pin below is exact up to rounding of O(N log N) terms


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return float(num / den) if den > 0 else float(num)


def _rng(seed):
    return np.random.default_rng(seed)


def _cvec(n, seed, batch=None):
    g = _rng(seed)
    shape = (n,) if batch is None else (batch, n)
    return g.uniform(-1, 1, shape) + 1j * g.uniform(-1, 1, shape)


# ---------------------------------------------------------------- 1D pins --

def pin_brute_force_1d(orc, sizes=(2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)):
    """Sec. 2 tree == Eq. E2 direct sum, and Sec. 3 inverse == Eq. E3 sum."""
    for n in sizes:
        x = _cvec(n, 1000 + n, batch=3)
        d = orc.dft(x)
        f = orc.fft(x)
        assert rel_l2(f, d) < TOL, f"fft vs direct DFT, N={n}: {rel_l2(f, d)}"
        assert rel_l2(orc.ifft(x), orc.idft(x)) < TOL, f"ifft vs direct IDFT, N={n}"


def pin_numpy_1d(orc, sizes=(2, 8, 64, 1024, 4096, 1 << 14)):
    """numpy.fft.fft(norm='forward') is Eq. E2; ifft(norm='forward') is Eq. E3."""
    for n in sizes:
        x = _cvec(n, 2000 + n, batch=2)
        assert rel_l2(orc.fft(x), np.fft.fft(x, norm="forward")) < TOL, f"fft vs numpy N={n}"
        assert rel_l2(orc.ifft(x), np.fft.ifft(x, norm="forward")) < TOL, f"ifft vs numpy N={n}"
    x = _cvec(37, 5)  # the direct sum takes any N
    assert rel_l2(orc.dft(x), np.fft.fft(x, norm="forward")) < TOL


def pin_closed_forms_1d(orc, n=64):
    j = np.arange(n)
    # delta at 0 -> every coefficient 1/N
    d0 = np.zeros(n, complex)
    d0[0] = 1
    assert np.allclose(orc.fft(d0), np.full(n, 1.0 / n), atol=1e-15, rtol=0)
    # delta at j0 -> exp(-2 pi i k j0 / N) / N
    j0 = 5
    dj = np.zeros(n, complex)
    dj[j0] = 1
    expect = np.array([complex(np.cos(2 * np.pi * k * j0 / n), -np.sin(2 * np.pi * k * j0 / n)) for k in range(n)]) / n
    assert np.allclose(orc.fft(dj), expect, atol=1e-15, rtol=0)
    # constant 1 -> c_0 = 1, the rest 0
    c = orc.fft(np.ones(n, complex))
    assert abs(c[0] - 1) < 1e-15 and np.max(np.abs(c[1:])) < 1e-15
    # cos(2 pi k0 j / N) -> 1/2 at k0 and N - k0
    k0 = 7
    c = orc.fft(np.cos(2 * np.pi * k0 * j / n).astype(complex))
    expect = np.zeros(n, complex)
    expect[k0] = expect[n - k0] = 0.5
    assert np.max(np.abs(c - expect)) < 1e-14
    # exp(+2 pi i k0 j / N) -> 1 at k0
    c = orc.fft(np.exp(2j * np.pi * k0 * j / n))
    expect = np.zeros(n, complex)
    expect[k0] = 1
    assert np.max(np.abs(c - expect)) < 1e-14
    # inverse of a single coefficient is the exponential polynomial itself
    e = np.zeros(n, complex)
    e[k0] = 1
    assert np.max(np.abs(orc.ifft(e) - np.exp(2j * np.pi * k0 * j / n))) < 1e-14


def pin_invariants_1d(orc, n=256):
    x = _cvec(n, 11)
    y = _cvec(n, 12)
    c = orc.fft(x)
    # Parseval with the 1/N forward scale: sum |c_k|^2 = (1/N) sum |f_j|^2
    assert abs(np.sum(np.abs(c) ** 2) - np.sum(np.abs(x) ** 2) / n) < 1e-12 * np.sum(np.abs(x) ** 2)
    # linearity
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    assert rel_l2(orc.fft(a * x + b * y), a * c + b * orc.fft(y)) < TOL
    # shift theorem: x[j - s] -> c_k exp(-2 pi i k s / N)
    s = 17
    k = np.arange(n)
    assert rel_l2(orc.fft(np.roll(x, s)), c * np.exp(-2j * np.pi * k * s / n)) < TOL
    # inverse(forward(f)) = f and forward(inverse(c)) = c
    assert rel_l2(orc.ifft(c), x) < TOL
    assert rel_l2(orc.fft(orc.ifft(x)), x) < TOL
    # real input -> c_{N-k} = conj(c_k)
    r = _rng(13).normal(size=n).astype(complex)
    cr = orc.fft(r)
    assert np.max(np.abs(cr[(n - k) % n] - np.conj(cr))) < 1e-15 * n
    # Sec. 3 reversal identity: inverse = N * forward, read in reverse order
    f = orc.ifft(x)
    assert rel_l2(f, n * c[(n - k) % n]) < TOL


def pin_bins(orc, n=1 << 12):
    x = _cvec(n, 21)
    bins = np.array([0, 1, 2, n // 2, n - 1, 1234])
    assert rel_l2(orc.dft_bins(x, bins), np.fft.fft(x, norm="forward")[bins]) < TOL
    assert rel_l2(orc.dft_bins(x, bins, inverse=True), np.fft.ifft(x, norm="forward")[bins]) < TOL


# ---------------------------------------------------------------- 2D pins --

def direct_dft2(f, sign=-1):
    """Unscaled 2D DFT by explicit exponent matrices (brute force, tiny only)."""
    rows, cols = f.shape
    u = np.arange(rows)
    v = np.arange(cols)
    Er = np.exp(sign * 2j * np.pi * np.outer(u, u) / rows)
    Ec = np.exp(sign * 2j * np.pi * np.outer(v, v) / cols)
    out = np.zeros((rows, cols), complex)
    for a in range(rows):
        for b in range(cols):
            out[a, b] = np.sum(f * Er[a][:, None] * Ec[b][None, :])
    return out


def pin_2d(orc, shapes=((4, 8), (8, 8), (16, 4), (2, 32))):
    for rows, cols in shapes:
        f = _cvec(cols, 31 + rows, batch=rows)
        pa = orc.fft2(f, 0)
        # brute-force definition, per-axis scale 1/(N M)
        assert rel_l2(pa, direct_dft2(f) / (rows * cols)) < TOL, (rows, cols)
        # Eq. 5 puts 1/N (N = rows) in front: M times the per-axis spectrum
        assert rel_l2(orc.fft2(f, 1), cols * pa) < TOL, (rows, cols)
        # Eq. 5's 2D-IDFT: (1/M) sum sum F e^{+...}
        F = _cvec(cols, 41 + rows, batch=rows)
        assert rel_l2(orc.ifft2(F, 1), direct_dft2(F, +1) / cols) < TOL
        assert rel_l2(orc.ifft2(F, 0), direct_dft2(F, +1)) < TOL
        for conv in (0, 1):
            assert rel_l2(orc.ifft2(orc.fft2(f, conv), conv), f) < TOL
    f = _cvec(64, 51, batch=32)
    assert rel_l2(orc.fft2(f, 0), np.fft.fft2(f, norm="forward")) < TOL
    assert rel_l2(orc.ifft2(f, 0), np.fft.ifft2(f, norm="forward")) < TOL


# ------------------------------------------------------------- pipeline --

def circular_filter_direct(img, H):
    """Convolution theorem written out: out = Re(h (*) img) with
    h = (1/(N M)) * unscaled inverse DFT of H, convolution by explicit sums."""
    rows, cols = img.shape
    h = direct_dft2(H.astype(complex), +1) / (rows * cols)
    out = np.zeros((rows, cols), complex)
    for a in range(rows):
        for b in range(cols):
            out += h[a, b] * np.roll(np.roll(img, a, axis=0), b, axis=1)
    return out.real


def pin_pipeline(orc):
    g = _rng(61)
    for rows, cols in ((8, 8), (16, 8), (4, 16)):
        img = g.normal(size=(rows, cols))
        H = g.uniform(0, 2, size=(rows, cols))  # no symmetry
        want = circular_filter_direct(img, H)
        for conv in (0, 1):
            assert rel_l2(orc.pipeline(img, H, conv), want) < TOL, (rows, cols, conv)
    img = g.normal(size=(3, 32, 16))
    # H == 1 is the identity
    assert rel_l2(orc.pipeline(img, np.ones((32, 16))), img) < TOL
    # H = delta at DC gives the image mean at every pixel
    d = np.zeros((32, 16))
    d[0, 0] = 1
    want = np.broadcast_to(img.mean(axis=(1, 2))[:, None, None], img.shape)
    assert rel_l2(orc.pipeline(img, d), want) < TOL
    # a Gaussian low-pass keeps a constant image constant (H[0,0] = 1)
    u = np.minimum(np.arange(32), 32 - np.arange(32))[:, None]
    v = np.minimum(np.arange(16), 16 - np.arange(16))[None, :]
    Hg = np.exp(-(u * u + v * v) / (2 * 3.0 ** 2))
    assert rel_l2(orc.pipeline(np.full((32, 16), 100.0), Hg), np.full((32, 16), 100.0)) < TOL
    # one filter per image == each image with its own filter
    Hs = g.uniform(0, 1, size=img.shape)
    each = np.stack([orc.pipeline(img[b], Hs[b]) for b in range(3)])
    assert rel_l2(orc.pipeline(img, Hs), each) < TOL


def pin_padded_pipeline(orc):
    """Zero padding to power-of-two sides, filter, crop (Sec. 5 application):
    brute force with the zeros written out by hand, identity and power-of-two
    special cases."""
    g = _rng(71)
    for (r, c), (R, C) in (((5, 6), (8, 8)), ((3, 7), (4, 8)), ((6, 3), (8, 4))):
        img = g.normal(size=(r, c))
        H = g.uniform(0, 2, size=(R, C))
        big = np.zeros((R, C))
        for i in range(r):
            for j in range(c):
                big[i, j] = img[i, j]
        want = circular_filter_direct(big, H)[:r, :c]
        got = orc.pipeline_padded(img, H)
        assert got.shape == (r, c) and rel_l2(got, want) < TOL, (r, c)
    img = g.normal(size=(2, 13, 21))
    assert rel_l2(orc.pipeline_padded(img, np.ones((16, 32))), img) < TOL  # H == 1
    img = g.normal(size=(16, 8))
    H = g.uniform(0, 2, size=(16, 8))
    assert rel_l2(orc.pipeline_padded(img, H), orc.pipeline(img, H)) < TOL  # nothing to pad
    # per-image filters on the padded grid
    img = g.normal(size=(3, 5, 6))
    Hs = g.uniform(0, 2, size=(3, 8, 8))
    each = np.stack([orc.pipeline_padded(img[b], Hs[b]) for b in range(3)])
    assert rel_l2(orc.pipeline_padded(img, Hs), each) < TOL


def pin_spectrum(orc):
    """Spectrum display |F| of the padded image: closed forms (delta, constant,
    one cosine), Parseval with the 1/(N M) scale, the Hermitian mirror, and
    Eq. 5's factor M."""
    R, C = 8, 16
    d = np.zeros((5, 11))
    d[0, 0] = 1
    s = orc.spectrum_padded(d, R, C)
    assert s.shape == (R, C) and np.max(np.abs(s - 1.0 / (R * C))) < 1e-15
    s = orc.spectrum_padded(np.full((5, 11), 3.0), R, C)
    assert abs(s[0, 0] - 3.0 * 55 / (R * C)) < 1e-14
    y, x = np.mgrid[0:R, 0:C]
    s = orc.spectrum_padded(np.cos(2 * np.pi * (2 * y / R + 3 * x / C)), R, C)
    want = np.zeros((R, C))
    want[2, 3] = want[R - 2, C - 3] = 0.5
    assert np.max(np.abs(s - want)) < 1e-14
    g = _rng(72)
    img = g.normal(size=(7, 13))
    s = orc.spectrum_padded(img, R, C)
    assert abs(np.sum(s * s) - np.sum(img * img) / (R * C)) < 1e-12 * np.sum(img * img)
    mirror = s[(-np.arange(R)) % R][:, (-np.arange(C)) % C]
    assert np.max(np.abs(s - mirror)) < 1e-14
    assert rel_l2(orc.spectrum_padded(img, R, C, 1), C * s) < TOL


def pin_pipeline_grad(orc, rows=8, cols=16, batch=2, probes=12):
    """Central finite differences of L = sum(y * G): the loss is linear in img
    (for fixed H) and in H (for fixed img), so the difference is exact up to
    rounding for any step."""
    g = _rng(71)
    img = g.normal(size=(batch, rows, cols))
    H = g.uniform(0, 2, size=(rows, cols))
    G = g.normal(size=(batch, rows, cols))
    gi, gh = orc.pipeline_grad(img, H, G)

    def loss(im, h):
        return float(np.sum(orc.pipeline(im, h) * G))

    for p in range(probes):
        b, r, c = g.integers(batch), g.integers(rows), g.integers(cols)
        e = np.zeros_like(img)
        e[b, r, c] = 1.0
        fd = (loss(img + e, H) - loss(img - e, H)) / 2.0
        assert abs(fd - gi[b, r, c]) < 1e-10 * (1 + abs(fd)), ("img", p, fd, gi[b, r, c])
        e = np.zeros_like(H)
        e[r, c] = 1.0
        fd = (loss(img, H + e) - loss(img, H - e)) / 2.0
        assert abs(fd - gh[r, c]) < 1e-10 * (1 + abs(fd)), ("H", p, fd, gh[r, c])


# ----------------------------------------------------- printed examples --

def read_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, n2, nlog, pfp, rsp = line.split()
            rows.append((int(n), int(n2), int(nlog), int(pfp), float(rsp)))
    return rows


def read_tree_n8():
    d = {"branch": {}}
    with open(os.path.join(GOLDEN, "tree_n8.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "branch":
                d["branch"][int(vals[0])] = [int(v) for v in vals[1:]]
            elif key == "leaves":
                d["leaves"] = [int(v) for v in vals]
            else:
                d[key] = int(vals[0])
    return d


def pin_table1(orc):
    for row in read_table1():
        assert orc.table1_row(row[0], 4) == row, (orc.table1_row(row[0], 4), row)


def pin_tree_example(orc):
    t = read_tree_n8()
    assert orc.tree_leaf_order(t["N"]) == t["leaves"]
    assert orc.table2_levels(t["N"], t["nproc"]) == (t["m"], t["m1"])
    assert orc.process_branches(t["N"], t["nproc"]) == dict(sorted(t["branch"].items()))


ALL_PINS = [
    pin_brute_force_1d,
    pin_numpy_1d,
    pin_closed_forms_1d,
    pin_invariants_1d,
    pin_bins,
    pin_2d,
    pin_pipeline,
    pin_pipeline_grad,
    pin_table1,
    pin_tree_example,
    pin_padded_pipeline,
    pin_spectrum,
]
