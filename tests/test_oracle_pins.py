"""Pins of the FP64 oracle (CPU only).

The oracle is the yardstick for every GPU parity test, so it is checked here
against facts that do not come from itself (see ``pins.py``), and the pins are
checked for teeth: each plausible mistake planted in a copy of the oracle must
make at least one pin fail.
"""

import types

import numpy as np
import pytest

import oracle
from tests import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    pin(oracle)


def _mutant(**overrides):
    m = types.SimpleNamespace(**{k: getattr(oracle, k) for k in dir(oracle) if not k.startswith("_")})
    for k, v in overrides.items():
        setattr(m, k, v)
    return m


def _last(x):
    return np.asarray(x).shape[-1]


MUTANTS = {
    # forward scale dropped (Eq. E2's 1/N missing)
    "fft_no_scale": dict(fft=lambda x: oracle.fft(x) * _last(x)),
    # forward exponent with the wrong sign
    "fft_wrong_sign": dict(fft=lambda x: np.conj(oracle.fft(np.conj(oracle._c128(x))))),
    # Sec. 3 inverse without the reversal (N * FFT read in order)
    "ifft_not_reversed": dict(ifft=lambda c: oracle.fft(c) * _last(c)),
    # inverse scaled by 1/N like the forward
    "ifft_scaled": dict(ifft=lambda c: oracle.ifft(c) / _last(c)),
    # a dropped term: the last sample ignored by the tree
    "fft_dropped_term": dict(fft=lambda x: oracle.fft(np.concatenate(
        [oracle._c128(x)[..., :-1], np.zeros_like(oracle._c128(x)[..., :1])], axis=-1))),
    # Eq. 5's "x M" step with the wrong axis length
    "eq5_wrong_axis": dict(fft2=lambda x, conv=0: oracle.fft2(x, 0) * (np.asarray(x).shape[-2] if conv else 1)),
    # transposed filter operand in the pipeline
    "pipeline_transposed_H": dict(pipeline=lambda img, H, conv=0: oracle.pipeline(img, np.swapaxes(H, -1, -2), conv)),
    # pipeline that forgets the imaginary part of the spectrum product
    "pipeline_real_only": dict(pipeline=lambda img, H, conv=0: np.real(oracle.ifft2(
        np.real(oracle.fft2(img, 0)) * H, 0))),
    # grad_H without the 1/s = N M factor
    "grad_H_unscaled": dict(pipeline_grad=lambda img, H, G: (
        oracle.pipeline_grad(img, H, G)[0], oracle.pipeline_grad(img, H, G)[1] / H.size)),
    # grad_img from the wrong operand (the image instead of the upstream gradient)
    "grad_img_wrong_operand": dict(pipeline_grad=lambda img, H, G: (
        oracle.pipeline(img, H), oracle.pipeline_grad(img, H, G)[1])),
    # Eq. multi summed from i = 0
    "multi_off_by_one": dict(table1_row=lambda n, nproc=4: (
        n, n * n, n * (n.bit_length() - 1),
        oracle.multiplications_parallel(n.bit_length() - 1, 2) + 2 ** (n.bit_length() - 3),
        oracle.table1_row(n, nproc)[4])),
    # leaves in natural order instead of bit-reversed
    "leaves_natural": dict(tree_leaf_order=lambda n: list(range(n))),
    # zeros put before the image (top-left) but the result cut from the top-left corner
    "pad_before_crop_after": dict(pipeline_padded=lambda img, H, conv=0: _pad_before(img, H, conv)),
    # result cut from the wrong corner of the padded grid
    "crop_wrong_corner": dict(pipeline_padded=lambda img, H, conv=0: np.asarray(oracle.pipeline(
        oracle.pad(img, *np.asarray(H).shape[-2:]), H, conv))[..., -np.shape(img)[-2]:, -np.shape(img)[-1]:]),
    # squared magnitude instead of sqrt(Re^2 + Im^2)
    "spectrum_squared": dict(spectrum_padded=lambda img, R, C, conv=0: oracle.spectrum_padded(img, R, C, conv) ** 2),
    # spectrum of the unscaled transform
    "spectrum_unscaled": dict(spectrum_padded=lambda img, R, C, conv=0: oracle.spectrum_padded(img, R, C, conv) * R * C),
}


def _pad_before(img, H, conv):
    img = np.asarray(img, dtype=np.float64)
    R, C = np.asarray(H).shape[-2:]
    r, c = img.shape[-2:]
    big = np.zeros(img.shape[:-2] + (R, C))
    big[..., R - r:, C - c:] = img
    return oracle.pipeline(big, H, conv)[..., :r, :c]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    m = _mutant(**MUTANTS[name])
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(m)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
