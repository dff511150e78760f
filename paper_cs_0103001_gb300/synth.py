"""Seeded synthetic inputs: star-field skies, random complex vectors, filters.

This module holds input generators only, none of the transform arithmetic, so
that the CUDA path and the FP64 oracle can be fed identical numbers.  Every
generator draws from ``numpy.random.default_rng(SeedSequence([103001, ...]))``
and returns float32 / complex64 arrays (the precision the GPU receives; the
oracle promotes the very same values to double).

Stand-in data: the paper filters a photograph of the galaxy NGC5194
(460 x 506 pixels, Sec. 5).  That image is not available, so a synthetic
sky of the same kind stands in: a flat background, Gaussian read noise and
point sources blurred by a Gaussian PSF.

Filters are real arrays H[u, v] in natural (unshifted) DFT index order, the
operator H: Z^2 -> R of Sec. 5.  Gaussian and Butterworth low-passes are the
workload's filters; :func:`disc_filter` is the paper's Eq. filtro.
"""

from __future__ import annotations

import numpy as np

SEED_ROOT = 103001


def rng_for(*tags: int) -> np.random.Generator:
    """Generator for a tag path, e.g. rng_for(cfg, image_index)."""
    return np.random.default_rng(np.random.SeedSequence([SEED_ROOT, *[int(t) for t in tags]]))


def sky(rows: int, cols: int, n_sources: int, *tags: int, background: float = 100.0,
        noise_sigma: float = 10.0, psf_sigma: float = 1.5, amp_log10=(1.0, 4.0),
        stamp_half: int = 8) -> np.ndarray:
    """Synthetic star field, float32 [rows, cols].

    background + N(0, noise_sigma^2) per pixel + ``n_sources`` Gaussian PSFs
    (sigma ``psf_sigma`` px) whose peak amplitude is log-uniform in
    10^amp_log10 and whose centre is uniform (sub-pixel) over the frame.
    Each stamp is truncated at +-``stamp_half`` px and clipped at the edges.
    """
    g = rng_for(*tags)
    img = background + noise_sigma * g.standard_normal((rows, cols))
    if n_sources > 0:
        amp = 10.0 ** g.uniform(amp_log10[0], amp_log10[1], n_sources)
        cy = g.uniform(0.0, rows, n_sources)
        cx = g.uniform(0.0, cols, n_sources)
        off = np.arange(-stamp_half, stamp_half + 1)
        iy = np.floor(cy).astype(np.int64)[:, None] + off[None, :]  # [K, S]
        ix = np.floor(cx).astype(np.int64)[:, None] + off[None, :]
        wy = np.exp(-((iy - cy[:, None]) ** 2) / (2.0 * psf_sigma ** 2))
        wx = np.exp(-((ix - cx[:, None]) ** 2) / (2.0 * psf_sigma ** 2))
        val = amp[:, None, None] * wy[:, :, None] * wx[:, None, :]  # [K, S, S]
        yy = np.broadcast_to(iy[:, :, None], val.shape)
        xx = np.broadcast_to(ix[:, None, :], val.shape)
        keep = (yy >= 0) & (yy < rows) & (xx >= 0) & (xx < cols)
        np.add.at(img, (yy[keep], xx[keep]), val[keep])
    return img.astype(np.float32)


def complex_uniform(shape, *tags: int) -> np.ndarray:
    """complex64 array whose real and imaginary parts are i.i.d. U[-1, 1]."""
    g = rng_for(*tags)
    re = g.uniform(-1.0, 1.0, shape)
    im = g.uniform(-1.0, 1.0, shape)
    return (re + 1j * im).astype(np.complex64)


def real_uniform(shape, *tags: int, low: float = -1.0, high: float = 1.0) -> np.ndarray:
    g = rng_for(*tags)
    return g.uniform(low, high, shape).astype(np.float32)


def wrapped_frequencies(n: int) -> np.ndarray:
    """Signed DFT bin of each index: k if k < n/2 else k - n (float64)."""
    k = np.arange(n, dtype=np.float64)
    return np.where(k < n / 2, k, k - n)


def _radius2(rows: int, cols: int) -> np.ndarray:
    u = wrapped_frequencies(rows)[:, None]
    v = wrapped_frequencies(cols)[None, :]
    return u * u + v * v


def gaussian_lowpass(rows: int, cols: int, sigma_bins: float) -> np.ndarray:
    """H = exp(-|k|^2 / (2 sigma^2)), |k| in bins of the wrapped frequencies."""
    return np.exp(-_radius2(rows, cols) / (2.0 * float(sigma_bins) ** 2)).astype(np.float32)


def butterworth_lowpass(rows: int, cols: int, order: int = 4, cutoff_frac: float = 0.1) -> np.ndarray:
    """H = 1 / (1 + (|k| / D0)^(2 order)) with D0 = cutoff_frac x Nyquist bins."""
    d0 = cutoff_frac * min(rows, cols) / 2.0
    r2 = _radius2(rows, cols)
    return (1.0 / (1.0 + (r2 / (d0 * d0)) ** order)).astype(np.float32)


def disc_filter(rows: int, cols: int, b: float) -> np.ndarray:
    """Eq. filtro: 0 where the distance of (u, v) from the centre (rows/2, cols/2)
    is at most b, 1 elsewhere.  In unshifted DFT order the centre is the
    highest frequency, so this removes high frequencies (a smoothing filter)."""
    u = np.arange(rows, dtype=np.float64)[:, None] - rows / 2.0
    v = np.arange(cols, dtype=np.float64)[None, :] - cols / 2.0
    return np.where(np.sqrt(u * u + v * v) <= b, 0.0, 1.0).astype(np.float32)


def random_filter(rows: int, cols: int, *tags: int) -> np.ndarray:
    """A real filter with no symmetry (values U[0, 2]), e.g. a learnt one."""
    return real_uniform((rows, cols), *tags, low=0.0, high=2.0)


def next_pow2(n: int) -> int:
    return 1 << max(0, int(n - 1).bit_length())


UNEVEN_SIDES = (64, 128, 256, 512, 1024, 2048)


def uneven_batch(count: int, *tags: int, sides=UNEVEN_SIDES, sigma_range=(8.0, 128.0),
                 sources_per_256sq: int = 50, min_sources: int = 5):
    """Images of mixed power-of-two sides, each with its own Gaussian low-pass.

    Returns a list of (img float32 [n, n], H float32 [n, n], sigma).  The side
    is drawn uniformly from ``sides``; the source count scales with the area
    (round(50 (n/256)^2), at least ``min_sources``).
    """
    g = rng_for(*tags)
    ns = g.choice(np.asarray(sides), size=count)
    sig = g.uniform(sigma_range[0], sigma_range[1], size=count)
    out = []
    for i, (n, s) in enumerate(zip(ns.tolist(), sig.tolist())):
        k = max(min_sources, int(round(sources_per_256sq * (n / 256.0) ** 2)))
        out.append((sky(n, n, k, *tags, 1 + i), gaussian_lowpass(n, n, s), s))
    return out
