"""Pins of the analytic transforms (App. B; Sec. "Bulk Fluid Method"; eq. potentialSolution)
against quadrature of the defining integrals, the printed k -> 0 limits and known limits."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import weights
from quadrature import ball_transform_radial, shell_transforms
from oracle.units import bjerrum_length_nm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "k0_limits.txt")


def eval_weights(kvec, R):
    kx, ky, kz = (np.array([[[v]]]) for v in kvec)
    w0, w1, w2, w3, wV1, wV2 = weights.fmt_weights_hat(kz, ky, kx, R)
    f = lambda a: complex(np.asarray(a).ravel()[0])
    return f(w0), f(w1), f(w2), f(w3), [f(v) for v in wV1], [f(v) for v in wV2]


@pytest.mark.parametrize("kvec", [(3.1, -1.7, 0.4), (0.05, 0.0, 0.02), (1.5, 1.0, -2.0), (10.0, 22.0, -7.5), (0.0, 0.0, 41.0)])
@pytest.mark.parametrize("R", [0.095, 0.181])
def test_fmt_weights_against_quadrature(kvec, R):
    k = np.array(kvec)
    kmag = np.linalg.norm(k)
    w0, w1, w2, w3, wV1, wV2 = eval_weights(kvec, R)
    shell, vec = shell_transforms(k, R)
    assert w2 == pytest.approx(shell, rel=1e-10, abs=1e-14)
    assert w0 == pytest.approx(shell / (4 * math.pi * R * R), rel=1e-10, abs=1e-14)
    assert w1 == pytest.approx(shell / (4 * math.pi * R), rel=1e-10, abs=1e-14)
    assert np.allclose(wV2, vec, rtol=1e-9, atol=1e-13)
    assert np.allclose(wV1, vec / (4 * math.pi * R), rtol=1e-9, atol=1e-13)
    ball = ball_transform_radial(kmag, R, lambda r: 1.0)
    assert w3.real == pytest.approx(ball, rel=1e-9, abs=1e-15)
    assert abs(w3.imag) == 0.0


def _golden_limits(R):
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, expr = line.split(None, 1)
            out[name] = eval(expr, {"pi": math.pi, "R": R})
    return out


@pytest.mark.parametrize("R", [0.095, 0.14, 0.5])
def test_k0_limits_printed_in_paper(R):
    lim = _golden_limits(R)
    w0, w1, w2, w3, wV1, wV2 = eval_weights((0.0, 0.0, 0.0), R)
    assert w0 == pytest.approx(lim["w0"])
    assert w1 == pytest.approx(lim["w1"])
    assert w2 == pytest.approx(lim["w2"])
    assert w3 == pytest.approx(lim["w3"])
    assert all(v == 0 for v in wV1) and all(v == 0 for v in wV2)
    # the closed forms approach the limits continuously
    w0e, w1e, w2e, w3e, _, _ = eval_weights((1e-4, 0.0, 0.0), R)
    assert w3e.real == pytest.approx(lim["w3"], rel=1e-6)
    b = weights.ball_integrals(np.array([0.0, 1e-3]), R)
    for name, arr in zip(("B_m1", "B_0", "B_1"), b):
        assert arr[0] == pytest.approx(lim[name], rel=1e-14)
        assert arr[1] == pytest.approx(lim[name], rel=1e-5)


@pytest.mark.parametrize("n,R", [(-1, 0.276), (0, 0.276), (1, 0.362)])
def test_ball_integrals_against_quadrature(n, R):
    for k in (0.3, 1.0, 1.5, 3.7, 25.0):
        val, _ = integrate.quad(lambda r: r ** (n + 1) * math.sin(k * r), 0.0, R, limit=400, epsabs=1e-15)
        b = weights.ball_integrals(np.array([k]), R)[n + 1][0]
        assert b == pytest.approx(4 * math.pi / k * val, rel=1e-10)


@pytest.mark.parametrize("k", [0.0, 0.5, 1.2, 1.9, 3.7, 19.0])
def test_delta_c_hat_is_transform_of_real_kernel(k):
    # Radial quadrature of eq. CplusPsiFunc; this fixes the prefactor of eq. CplusPsiHat.
    lb = bjerrum_length_nm(298.15, 78.5)
    zi, zj, li, lj = 1.0, -1.0, 0.4, 0.55
    Rij = 0.276
    kern = lambda r: float(weights.delta_c_real(r, zi, zj, li, lj, Rij, lb))
    if k == 0.0:
        quad, _ = integrate.quad(lambda r: 4 * math.pi * r * r * kern(r), 0, Rij, limit=200)
    else:
        quad = ball_transform_radial(k, Rij, kern)
    got = weights.delta_c_hat(np.array([k]), zi, zj, li, lj, Rij, lb)[0]
    assert got == pytest.approx(quad, rel=1e-9)


def test_delta_c_coulomb_limit():
    # Gamma -> 0 makes lambda -> infinity: the kernel tends to the Coulomb term lambda_B z_i z_j / r.
    lb = 0.714
    r = np.linspace(0.05, 0.3, 7)
    big = 1e9
    val = weights.delta_c_real(r, 2.0, -1.0, big, big * 1.0000001, 0.3, lb)
    assert np.allclose(val, lb * 2.0 * -1.0 / r, rtol=1e-6)


def test_laplacian_symbol_is_stencil_eigenvalue():
    # The 7-point FD Laplacian applied to a grid plane wave multiplies it by -symbol.
    shape = (6, 8, 10)
    h = (0.1, 0.07, 0.13)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for jx, jy, jz in [(1, 2, 3), (5, 4, 3), (0, 0, 1)]:
        kx = 2 * math.pi * jx / (nx * h[0])
        ky = 2 * math.pi * jy / (ny * h[1])
        kz = 2 * math.pi * jz / (nz * h[2])
        f = np.exp(1j * (kx * x * h[0] + ky * y * h[1] + kz * z * h[2]))
        lap = sum((np.roll(f, 1, a) - 2 * f + np.roll(f, -1, a)) / hd ** 2
                  for a, hd in ((2, h[0]), (1, h[1]), (0, h[2])))
        sym = weights.laplacian_symbol(np.array(kz), np.array(ky), np.array(kx), h)
        assert np.allclose(-lap, sym * f, atol=1e-9)
