"""Grid wave vectors and the 3D discrete Fourier transform (test infrastructure only).

Fields are arrays indexed [..., z, y, x] (x fastest), on a periodic box with
N_d points of spacing h_d per axis, x_j = j h_d and L_d = N_d h_d.  App. B prints
h_d = L_d / (N_d - 1), the non-periodic convention; for periodic grids the
spacing is read as L_d / N_d and h_d is given directly.

Wave vectors follow eq. Kvalues: k_d = 2 pi j / (N_d h_d) for j <= N_d / 2 and
-2 pi (N_d - j) / (N_d h_d) otherwise.

The transform is the definition written out:
    forward   F[j] = sum_m f[m] exp(-2 pi i sum_d j_d m_d / N_d)
    inverse   f[m] = (1/N) sum_j F[j] exp(+2 pi i sum_d j_d m_d / N_d)
The 3D exponential factorises over axes, so ``dft3`` applies one explicit
N_d x N_d DFT matrix per axis (a matrix product, O(N sum N_d)).
``dft3_bruteforce`` is the unfactorised triple sum, O(N^2), for tiny grids.

Parity: pinned by tests/test_oracle_fourier.py against the brute-force sum,
against numpy.fft (a library routine used only in that test), and against
transforms known in closed form (delta, single Fourier mode).
"""

import math

import numpy as np


def wavenumbers(n: int, h: float) -> np.ndarray:
    """k_d for j = 0..n-1 per eq. Kvalues."""
    j = np.arange(n)
    k = np.where(j <= n / 2, 2.0 * math.pi * j / (n * h), -2.0 * math.pi * (n - j) / (n * h))
    return k.astype(np.float64)


def kgrid(shape, h):
    """Broadcastable (kz, ky, kx) arrays for a field of shape (Nz, Ny, Nx) and spacing (hx, hy, hz)."""
    nz, ny, nx = shape
    hx, hy, hz = h
    kx = wavenumbers(nx, hx)[None, None, :]
    ky = wavenumbers(ny, hy)[None, :, None]
    kz = wavenumbers(nz, hz)[:, None, None]
    return kz, ky, kx


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """M[j, m] = exp(sign * 2 pi i (j m mod n) / n)."""
    j = np.arange(n)
    jm = np.outer(j, j) % n
    return np.exp(sign * 2j * math.pi * jm / n)


def _apply_axis(f, mat, axis):
    f = np.moveaxis(f, axis, -1)
    g = f @ mat.T
    return np.moveaxis(g, -1, axis)


def dft3(f):
    """Forward 3D DFT over the last three axes (z, y, x)."""
    g = np.asarray(f, dtype=np.complex128)
    for axis in (-1, -2, -3):
        g = _apply_axis(g, dft_matrix(g.shape[axis], -1), axis)
    return g


def idft3(F):
    """Inverse 3D DFT over the last three axes, with the 1/N factor."""
    g = np.asarray(F, dtype=np.complex128)
    n = g.shape[-1] * g.shape[-2] * g.shape[-3]
    for axis in (-1, -2, -3):
        g = _apply_axis(g, dft_matrix(g.shape[axis], +1), axis)
    return g / n


def dft3_bruteforce(f, sign=-1):
    """Unfactorised 3D DFT sum over all (j, m) pairs (tiny grids only)."""
    f = np.asarray(f, dtype=np.complex128)
    nz, ny, nx = f.shape
    mz, my, mx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mz, my, mx = mz.ravel(), my.ravel(), mx.ravel()
    flat = f.ravel()
    out = np.empty(f.size, dtype=np.complex128)
    for idx in range(f.size):
        jz, jy, jx = mz[idx], my[idx], mx[idx]
        phase = (jz * mz / nz + jy * my / ny + jx * mx / nx)
        out[idx] = np.sum(flat * np.exp(sign * 2j * math.pi * phase))
    return out.reshape(f.shape)
