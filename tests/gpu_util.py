"""Shared helpers for the GPU parity tests."""

import math

import numpy as np

FP32_PER_LEVEL = 2e-7  # tolerance 2e-7 * log2(N), N = points of one transform
FP64_TOL = 1e-12


def tol_fp32(points: int) -> float:
    return FP32_PER_LEVEL * math.log2(points)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / den) if den > 0 else float(np.linalg.norm(a.ravel()))


def max_rel_l2(a, b, axes) -> float:
    """Largest relative L2 error over the leading (batch) index, norms over `axes`."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=axes))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=axes))
    den = np.where(den > 0, den, 1.0)
    return float(np.max(num / den))
