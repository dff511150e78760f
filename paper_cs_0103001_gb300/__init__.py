"""gbfft: GB300-native (sm_103a) FFT -> filter -> IFFT library.

Implements the transforms of Higuera, Sarria, Fonseca and Idarraga,
"Construction of an algorithm in parallel for the Fast Fourier Transform"
(arXiv cs/0103001): the 1/N-normalised forward DFT (Eq. E2), its unscaled
inverse (Eq. E3), the row-column 2D transform (Sec. 4) and the image filter
application (Sec. 5), as hand-written CUDA kernels behind a C ABI
(include/gbfft.h, libgbfft.so).  PyTorch is used for device memory and
streams only.

Importing this package loads libgbfft.so and fails if it is missing; build it
with ``paper_cs_0103001_gb300.build.build()``.
"""

from .api import (  # noqa: F401
    Plan1D,
    Plan2D,
    Plan2DBatched,
    clear_plan_cache,
    fft,
    fft2_filter_ifft2,
    fft2_filter_ifft2_analytic,
    fft2_filter_ifft2_batched,
    fft2_filter_ifft2_padded,
    fft2_spectrum,
    ifft,
)

__all__ = ["fft", "ifft", "fft2_filter_ifft2", "fft2_filter_ifft2_analytic", "fft2_filter_ifft2_batched",
           "fft2_filter_ifft2_padded",
           "fft2_spectrum", "Plan1D", "Plan2D", "Plan2DBatched", "clear_plan_cache"]
