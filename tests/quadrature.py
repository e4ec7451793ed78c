"""Quadrature of the paper's defining integrals, used to pin the oracle's closed forms."""
import math

import numpy as np
from scipy import integrate


def sphere_quadrature(nu=96, nphi=192):
    """Nodes (unit vectors) and weights for integrals over the unit sphere."""
    u, wu = np.polynomial.legendre.leggauss(nu)
    phi = 2 * math.pi * np.arange(nphi) / nphi
    U, P = np.meshgrid(u, phi, indexing="ij")
    st = np.sqrt(1 - U * U)
    nodes = np.stack([st * np.cos(P), st * np.sin(P), U], axis=-1).reshape(-1, 3)
    w = (wu[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    return nodes, w


def shell_transforms(k, R):
    """int delta(|r|-R) e^{-ik.r} d^3r and int (r/|r|) delta(|r|-R) e^{-ik.r} d^3r (eq. omegaDef)."""
    nodes, w = sphere_quadrature()
    ph = np.exp(-1j * R * nodes @ np.asarray(k, dtype=float))
    scalar = R * R * np.sum(w * ph)
    vector = R * R * np.sum((w * ph)[:, None] * nodes, axis=0)
    return scalar, vector


def ball_transform_radial(kmag, R, func):
    """int_{|r|<=R} func(|r|) e^{-ik.r} d^3r = 4 pi int_0^R r^2 func(r) sin(kr)/(kr) dr."""
    if kmag == 0.0:
        val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * func(r), 0.0, R, limit=400)
        return val
    val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * func(r) * math.sin(kmag * r) / (kmag * r),
                            0.0, R, limit=400, epsabs=1e-14, epsrel=1e-12)
    return val


def fmt_transforms_by_quadrature(k, R):
    """(w0, w1, w2, w3, wV1[3], wV2[3]) at wave vector k (x, y, z) from the defining integrals."""
    shell, vec = shell_transforms(k, R)
    ball = ball_transform_radial(float(np.linalg.norm(k)), R, lambda r: 1.0)
    return (shell / (4 * math.pi * R * R), shell / (4 * math.pi * R), shell, ball,
            vec / (4 * math.pi * R), vec)
