"""gbfft: GB300-native (sm_103a) FFT -> filter -> IFFT library.

Implements the transforms of Higuera, Sarria, Fonseca and Idarraga,
"Construction of an algorithm in parallel for the Fast Fourier Transform"
(arXiv cs/0103001): the 1/N-normalised forward DFT (Eq. E2), its unscaled
inverse (Eq. E3), the row-column 2D transform (Sec. 4) and the image filter
application (Sec. 5), as hand-written CUDA kernels behind a C ABI
(include/gbfft.h, libgbfft.so).  PyTorch is used for device memory and
streams only.

The transforms load libgbfft.so on first use (the first attribute taken from
this package other than ``synth``) and raise if it is missing; build it with
``paper_cs_0103001_gb300.build.build()``.  ``synth`` (seeded input
generators, no transform arithmetic) and ``slab`` (index maps of the row-slab
decomposition) import without the library, so a process that only generates
inputs maps no CUDA code.
"""

import importlib

__all__ = ["fft", "ifft", "fft2_filter_ifft2", "fft2_filter_ifft2_analytic", "fft2_filter_ifft2_batched",
           "fft2_filter_ifft2_padded", "fft2_filter_ifft2_sharded", "fft2_spectrum", "Plan1D", "Plan2D",
           "Plan2DBatched", "Plan2DSlab", "clear_plan_cache", "measure_fma_peak"]


def __getattr__(name):
    if name in __all__:
        return getattr(importlib.import_module(".api", __name__), name)
    if name in ("api", "_native", "slab"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
