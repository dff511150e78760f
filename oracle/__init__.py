"""FP64 CPU oracle for the FFT -> filter -> IFFT path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark are the only code that may import this package.  The
product library never loads it, and it shares no code with the CUDA kernels.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double), compiled on first
use with gcc into ``liboracle.so`` next to it.  This module only marshals
numpy arrays in and out, plus a few tiny pure-Python restatements of the
paper's bookkeeping (the tree's leaf order, the per-process branches and the
multiplication-count model of Sec. 3, Eq. multi, Table 1).

Inputs are promoted to float64/complex128 before the C code sees them; the
GPU receives the same values in float32/complex64, so both sides start from
identical numbers.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PER_AXIS = 0  # 1D definition on each axis: 1/M on rows, 1/N on columns
PAPER_EQ5 = 1  # Eq. 5: (1/N) in front, built as row FFT -> x M -> column FFT


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc -O3 -fopenmp (plain C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int64
            for name, args in {
                "orc_dft": [P, P, I, I],
                "orc_idft": [P, P, I, I],
                "orc_fft": [P, P, I, I],
                "orc_ifft": [P, P, I, I],
                "orc_dft_bins": [P, I, P, I, ctypes.c_int, P],
                "orc_fft2": [P, P, I, I, I, ctypes.c_int],
                "orc_ifft2": [P, P, I, I, I, ctypes.c_int],
                "orc_pipeline": [P, P, P, I, I, I, I, ctypes.c_int],
                "orc_pipeline_grad": [P, P, P, P, P, I, I, I],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (batch, rows and columns)."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (status {rc})")


def _batched_1d(fn: str, x) -> np.ndarray:
    x = _c128(x)
    if x.ndim == 0:
        raise ValueError("need at least one dimension")
    n = x.shape[-1]
    batch = x.size // n if n else 0
    y = np.empty_like(x)
    _check(getattr(_load(), fn)(_ptr(x), _ptr(y), n, batch), fn)
    return y


def dft(x) -> np.ndarray:
    """Eq. E2 as the O(N^2) sum along the last axis: c_k = (1/N) sum_j f_j e^{-2 pi i kj/N}."""
    return _batched_1d("orc_dft", x)


def idft(c) -> np.ndarray:
    """Eq. E3 at x_j = 2 pi j/N as the O(N^2) sum: f_j = sum_k c_k e^{+2 pi i kj/N} (no scale)."""
    return _batched_1d("orc_idft", c)


def fft(x) -> np.ndarray:
    """Sec. 2 radix-2 tree (decimation in time) with the Eq. E2 1/N; N = 2^m, m >= 1."""
    return _batched_1d("orc_fft", x)


def ifft(c) -> np.ndarray:
    """Sec. 3 inverse: N * FFT(c) read in reverse order, f_k = N FFT(c)[(N-k) mod N]."""
    return _batched_1d("orc_ifft", c)


def dft_bins(x, bins, inverse: bool = False) -> np.ndarray:
    """Eq. E2 (or Eq. E3 if ``inverse``) at the listed bins of one 1D transform, O(N) each."""
    x = _c128(x).reshape(-1)
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64).reshape(-1))
    y = np.empty(b.size, dtype=np.complex128)
    _check(_load().orc_dft_bins(_ptr(x), x.size, _ptr(b), b.size, int(bool(inverse)), _ptr(y)), "dft_bins")
    return y


def _batched_2d(fn: str, x, conv: int) -> np.ndarray:
    x = _c128(x)
    if x.ndim < 2:
        raise ValueError("need at least two dimensions")
    rows, cols = x.shape[-2:]
    batch = x.size // (rows * cols) if rows * cols else 0
    y = np.empty_like(x)
    _check(getattr(_load(), fn)(_ptr(x), _ptr(y), rows, cols, batch, int(conv)), fn)
    return y


def fft2(x, conv: int = PER_AXIS) -> np.ndarray:
    """Sec. 4: FFT on rows, then on columns, over the last two axes (rows x cols)."""
    return _batched_2d("orc_fft2", x, conv)


def ifft2(x, conv: int = PER_AXIS) -> np.ndarray:
    """Inverse of :func:`fft2` in the same convention."""
    return _batched_2d("orc_ifft2", x, conv)


def pipeline(img, H, conv: int = PER_AXIS) -> np.ndarray:
    """Sec. 5: Re(ifft2(H * fft2(img))).

    ``img`` is [..., rows, cols] real; ``H`` is [rows, cols] (shared) or has the
    same shape as ``img`` (one filter per image).  Returns float64.
    """
    img = _f64(img)
    H = _f64(H)
    rows, cols = img.shape[-2:]
    batch = img.size // (rows * cols)
    if H.shape == (rows, cols):
        h_stride = 0
    elif H.shape == img.shape:
        h_stride = rows * cols
    else:
        raise ValueError(f"filter shape {H.shape} does not match image shape {img.shape}")
    out = np.empty_like(img)
    _check(_load().orc_pipeline(_ptr(img), _ptr(H), _ptr(out), rows, cols, batch, h_stride, int(conv)), "pipeline")
    return out


def pipeline_grad(img, H, G):
    """Gradients of ``pipeline`` for an upstream gradient G = dL/dy.

    Returns (grad_img, grad_H); H is shared by the batch and grad_H is summed
    over it.  Closed forms: grad_img = pipeline(G, H);
    grad_H[k] = N M sum_b Re(conj(fft2(G_b)[k]) fft2(img_b)[k]).
    """
    img = _f64(img)
    H = _f64(H)
    G = _f64(G)
    rows, cols = img.shape[-2:]
    if H.shape != (rows, cols) or G.shape != img.shape:
        raise ValueError("shape mismatch")
    batch = img.size // (rows * cols)
    gi = np.empty_like(img)
    gh = np.empty_like(H)
    _check(_load().orc_pipeline_grad(_ptr(img), _ptr(H), _ptr(G), _ptr(gi), _ptr(gh), rows, cols, batch),
           "pipeline_grad")
    return gi, gh


def spectrum(F) -> np.ndarray:
    """Sec. 5 spectrum display value sqrt(Re^2 + Im^2) of a transform."""
    F = _c128(F)
    return np.sqrt(F.real * F.real + F.imag * F.imag)


# --------------------------------------------------------------------------
# Sec. 5's application path for an image whose sides are not powers of two:
# the image is enlarged with zeros to power-of-two sides before the transform,
# and the filtered result is cut back to the original size.  Where the zeros
# go is not stated; they are appended after the last row and the last column.
# --------------------------------------------------------------------------

def pad(img, rows: int, cols: int) -> np.ndarray:
    """Zero-extend [..., r, c] to [..., rows, cols] (zeros after the last row
    and after the last column); float64."""
    img = np.asarray(img, dtype=np.float64)
    r, c = img.shape[-2:]
    if r > rows or c > cols:
        raise ValueError("image larger than the padded size")
    out = np.zeros(img.shape[:-2] + (rows, cols))
    out[..., :r, :c] = img
    return out


def crop(x, rows: int, cols: int) -> np.ndarray:
    """The first `rows` rows and `cols` columns of [..., R, C]."""
    return np.array(np.asarray(x)[..., :rows, :cols])


def pipeline_padded(img, H, conv: int = PER_AXIS) -> np.ndarray:
    """Sec. 5 on a zero-padded image: crop(pipeline(pad(img), H)).  H is given
    on the padded grid ([R, C] shared, or [..., R, C] per image)."""
    img = np.asarray(img, dtype=np.float64)
    R, C = np.asarray(H).shape[-2:]
    return crop(pipeline(pad(img, R, C), H, conv), img.shape[-2], img.shape[-1])


def spectrum_padded(img, rows: int, cols: int, conv: int = PER_AXIS) -> np.ndarray:
    """Sec. 5 spectrum display of the zero-padded image: |fft2(pad(img))| on
    the rows x cols grid, in natural (unshifted) order."""
    return spectrum(fft2(pad(img, rows, cols), conv))


# --------------------------------------------------------------------------
# The paper's bookkeeping (pure Python, tiny inputs only).
# --------------------------------------------------------------------------

def tree_leaf_order(n: int) -> list[int]:
    """Sample index at each leaf of the Sec. 2 tree, left to right.

    A node holding a subsequence sends its even-position samples to the left
    child and its odd-position samples to the right child, down to single
    samples.
    """
    def leaves(seq):
        if len(seq) == 1:
            return list(seq)
        return leaves(seq[0::2]) + leaves(seq[1::2])

    if n < 1 or n & (n - 1):
        raise ValueError("n must be a power of two")
    return leaves(list(range(n)))


def process_branches(n: int, nproc: int) -> dict[int, list[int]]:
    """Samples each process owns in Sec. 2's distribution: the leaves of its
    own subtree, i.e. every sample j with j mod nproc == idproc."""
    if nproc < 1 or nproc & (nproc - 1) or n % nproc:
        raise ValueError("nproc must be a power of two dividing n")
    order = tree_leaf_order(n)
    width = n // nproc
    # the subtree under level m1 = m - log2(nproc) covers `width` adjacent leaves
    branches = {}
    for s in range(nproc):
        leaf_block = order[s * width:(s + 1) * width]
        branches[leaf_block[0] % nproc] = leaf_block
    return dict(sorted(branches.items()))


def table2_levels(n: int, nproc: int) -> tuple[int, int]:
    """Table 2's m = log2 N and m1 = m - log2(nproc) (the last level every process works)."""
    m = n.bit_length() - 1
    l = nproc.bit_length() - 1
    if 1 << m != n or 1 << l != nproc:
        raise ValueError("powers of two only")
    return m, m - l


def multiplications_parallel(m: int, l: int) -> int:
    """Eq. multi: (m-l) 2^(m-l) + sum_{i=1..l} 2^(m-l+i) products per processor path."""
    if m < 1 or l < 0 or l > m:
        raise ValueError("need 0 <= l <= m, m >= 1")
    return (m - l) * 2 ** (m - l) + sum(2 ** (m - l + i) for i in range(1, l + 1))


def speedup_ratio(m: int, l: int) -> float:
    """Sec. 3 ratio of sequential (N log2 N = m 2^m) to parallel products."""
    return m * 2 ** m / multiplications_parallel(m, l)


def table1_row(n: int, nproc: int = 4) -> tuple[int, int, int, int, float]:
    """One row of Table 1: N, N^2, N log2 N, Pfp, RSP (RSP rounded to 2 places)."""
    m = n.bit_length() - 1
    l = nproc.bit_length() - 1
    return n, n * n, n * m, multiplications_parallel(m, l), round(speedup_ratio(m, l), 2)
