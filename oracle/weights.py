"""Analytic Fourier transforms used by the convolutions (test infrastructure only).

Transforms are  w_hat(k) = integral w(r) exp(-i k . r) d^3 r  (App. B).

FMT weights of a sphere of radius R (eq. omegaDef), with x = |k| R:
    w2_hat  = 4 pi R sin(x) / |k|                             eq. OmegaHat2
    w0_hat  = sin(x) / x,   w1_hat = sin(x) / |k|              eq. omegaHat0and1
    w3_hat  = 4 pi (sin x - x cos x) / |k|^3                   eq. omegaHat3
    wV2_hat = -4 pi i (sin x - x cos x) / |k|^2 * k / |k|      eq. omegaHatV2
    wV1_hat = wV2_hat / (4 pi R)                               eq. omegaDef
with the k -> 0 limits 1, R, 4 pi R^2, 4 pi R^3 / 3, 0, 0 printed at the end of
App. B.

Bulk-fluid kernel (Sec. "Bulk Fluid Method"): the real-space MSA kernel
eq. CplusPsiFunc, in kT units,
    DC_ij(r) = (lambda_B z_i z_j / 2) [ r/(2 l_i l_j) - (l_i + l_j)/(l_i l_j)
               + ((l_i - l_j)^2/(2 l_i l_j) + 2) / r ]   for r <= R_ij = R_i + R_j,
and 0 beyond, with l_k = R_k + 1/(2 Gamma).  Its transform is built from the
ball integrals (4 pi / k) I_n, n = -1, 0, 1, printed in that section:
    DC_ij_hat = (lambda_B z_i z_j / 2) (4 pi / k) [ I_1/(2 l_i l_j)
                - (l_i + l_j)/(l_i l_j) I_0 + ((l_i - l_j)^2/(2 l_i l_j) + 2) I_-1 ].
eq. CplusPsiHat prints the prefactor z_i z_j e^2 / (eps |k|), twice what the
real-space kernel gives (z_i z_j e^2 / (8 pi eps) times 4 pi / k); the
real-space kernel is taken as the definition, so the prefactor is
2 pi lambda_B z_i z_j / k.  R in I_n is the integration radius R_ij.

Small |k|R: the printed closed forms cancel catastrophically as |k|R -> 0 (the
paper itself takes the limit by Taylor expansion).  Below y = |k|R = 0.5 the
oracle sums the power series of the defining integral instead,
    (4 pi / k) I_n = 4 pi R^(n+3) sum_m (-1)^m y^(2m) / ((2m+1)! (2m+n+3)),
obtained by expanding sin(k r) in int_0^R r^(n+1) sin(k r) dr.  (sin x - x cos x)/x^3
in the FMT weights is the n = 0 case divided by 4 pi R^3.

Poisson symbol (eq. potentialSolution): the eigenvalues of the 7-point FD
Laplacian, sum_d 2 (1 - cos(k_d h_d)) / h_d^2 (the printed "cos k_x" is read
as cos(k_x h_x)).

Parity: pinned by tests/test_oracle_weights.py against 1D radial and 2D
spherical quadrature of the defining integrals, the printed k -> 0 limits
(tests/golden/k0_limits.txt), and the Coulomb limit of the MSA kernel.
"""

import math

import numpy as np


SERIES_CUTOFF = 0.5


def _ball_series(y, n, terms=10):
    """sum_m (-1)^m y^(2m) / ((2m+1)! (2m+n+3))."""
    acc = np.zeros_like(y)
    fact = 1.0
    for m in range(terms):
        if m > 0:
            fact *= (2 * m) * (2 * m + 1)
        acc = acc + (-1) ** m * y ** (2 * m) / (fact * (2 * m + n + 3))
    return acc


def _sinc3(x):
    """(sin x - x cos x) / x^3, with the series below SERIES_CUTOFF (value 1/3 at 0)."""
    xs = np.where(x < SERIES_CUTOFF, 1.0, x)
    direct = (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(x < SERIES_CUTOFF, _ball_series(x, 0), direct)


def fmt_weights_hat(kz, ky, kx, radius):
    """w_hat^alpha(k) for one species.

    Returns (w0, w1, w2, w3, wV1, wV2) where the scalars are real arrays and
    wV1, wV2 are lists of three complex arrays ordered (x, y, z).
    """
    R = float(radius)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    kmag = np.broadcast_to(kmag, np.broadcast_shapes(kx.shape, ky.shape, kz.shape))
    zero = kmag == 0.0
    ks = np.where(zero, 1.0, kmag)          # placeholder where k = 0 (limit used there)
    x = ks * R
    s, c = np.sin(x), np.cos(x)
    w2 = np.where(zero, 4.0 * math.pi * R * R, 4.0 * math.pi * R * s / ks)
    w0 = np.where(zero, 1.0, s / x)
    w1 = np.where(zero, R, s / ks)
    j = _sinc3(np.where(zero, 0.0, x))
    w3 = 4.0 * math.pi * R ** 3 * j                    # = 4 pi (sin x - x cos x) / |k|^3
    radial = np.where(zero, 0.0, -4.0 * math.pi * R * R * x * j)   # = -4 pi (sin x - x cos x)/|k|^2, times i k_hat
    wV2 = [1j * radial * np.broadcast_to(kd, kmag.shape) / ks for kd in (kx, ky, kz)]
    wV1 = [w / (4.0 * math.pi * R) for w in wV2]
    return w0, w1, w2, w3, wV1, wV2


def ball_integrals(kmag, R):
    """(4 pi / k) I_n for n = -1, 0, 1 (Sec. "Bulk Fluid Method") with their k -> 0 limits."""
    kmag = np.asarray(kmag, dtype=np.float64)
    y = kmag * R
    small = y < SERIES_CUTOFF
    k = np.where(small, 1.0, kmag)
    s, c = np.sin(k * R), np.cos(k * R)
    i_m1 = (1.0 - c) / k
    i_0 = -R * c / k + s / k ** 2
    i_1 = -R * R * c / k + 2.0 * R * s / k ** 2 - 2.0 * (1.0 - c) / k ** 3
    f = 4.0 * math.pi / k
    b_m1 = np.where(small, 4.0 * math.pi * R ** 2 * _ball_series(y, -1), f * i_m1)
    b_0 = np.where(small, 4.0 * math.pi * R ** 3 * _ball_series(y, 0), f * i_0)
    b_1 = np.where(small, 4.0 * math.pi * R ** 4 * _ball_series(y, 1), f * i_1)
    return b_m1, b_0, b_1


def delta_c_real(r, zi, zj, li, lj, Rij, lb):
    """Real-space kernel DC_ij(r) in kT units (eq. CplusPsiFunc), 0 for r > R_ij."""
    r = np.asarray(r, dtype=np.float64)
    val = 0.5 * lb * zi * zj * (r / (2.0 * li * lj) - (li + lj) / (li * lj)
                                + ((li - lj) ** 2 / (2.0 * li * lj) + 2.0) / r)
    return np.where(r <= Rij, val, 0.0)


def delta_c_hat(kmag, zi, zj, li, lj, Rij, lb):
    """Transform of delta_c_real (see module docstring for the prefactor reading)."""
    b_m1, b_0, b_1 = ball_integrals(kmag, Rij)
    if np.isinf(li) and np.isinf(lj):
        # Gamma = 0 (no ions in the bath): l -> infinity leaves the Coulomb term lambda_B z_i z_j / r
        return lb * zi * zj * b_m1
    return 0.5 * lb * zi * zj * (b_1 / (2.0 * li * lj) - (li + lj) / (li * lj) * b_0
                                 + ((li - lj) ** 2 / (2.0 * li * lj) + 2.0) * b_m1)


def laplacian_symbol(kz, ky, kx, h):
    """sum_d 2 (1 - cos(k_d h_d)) / h_d^2, the FD-Laplacian eigenvalues of eq. potentialSolution."""
    hx, hy, hz = h
    return (2.0 * (1.0 - np.cos(kx * hx)) / hx ** 2
            + 2.0 * (1.0 - np.cos(ky * hy)) / hy ** 2
            + 2.0 * (1.0 - np.cos(kz * hz)) / hz ** 2)
