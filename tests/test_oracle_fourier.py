"""Pins of the oracle's wave vectors (eq. Kvalues) and explicit DFT."""
import math

import numpy as np
import pytest

from oracle import fourier


@pytest.mark.parametrize("n", [5, 8, 12, 16])
def test_wavenumbers_match_eq_kvalues(n):
    h = 0.07
    k = fourier.wavenumbers(n, h)
    ref = 2 * math.pi * np.fft.fftfreq(n, d=h)     # library ordering, Nyquist negative
    for j in range(n):
        if 2 * j == n:
            assert k[j] == pytest.approx(math.pi / h)   # eq. Kvalues: j <= N/2 is positive
        else:
            assert k[j] == pytest.approx(ref[j], abs=1e-12)


def test_separable_equals_bruteforce():
    rng = np.random.default_rng(0)
    f = rng.standard_normal((4, 6, 5)) + 1j * rng.standard_normal((4, 6, 5))
    assert np.allclose(fourier.dft3(f), fourier.dft3_bruteforce(f, -1), atol=1e-11)
    assert np.allclose(fourier.idft3(f) * f.size, fourier.dft3_bruteforce(f, +1), atol=1e-11)


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 9), (3, 16, 10), (161, 21, 21), (35, 22, 23)])
def test_dft_matches_library_fft(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((2,) + shape)
    F = fourier.dft3(f)
    assert np.allclose(F, np.fft.fftn(f, axes=(-3, -2, -1)), atol=1e-10)
    assert np.allclose(fourier.idft3(F), f, atol=1e-13)


def test_delta_and_single_mode():
    shape = (6, 8, 10)
    d = np.zeros(shape)
    d[0, 0, 0] = 1.0
    assert np.allclose(fourier.dft3(d), 1.0)
    # cos(2 pi (2 x/Nx + 1 y/Ny)) -> N/2 at (jz, jy, jx) = (0, 1, 2) and (0, Ny-1, Nx-2)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.cos(2 * math.pi * (2 * x / nx + y / ny))
    F = fourier.dft3(f)
    expect = np.zeros(shape, dtype=complex)
    expect[0, 1, 2] = expect[0, ny - 1, nx - 2] = f.size / 2
    assert np.allclose(F, expect, atol=1e-10)
