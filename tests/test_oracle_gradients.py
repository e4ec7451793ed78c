"""Pins of the grand-potential gradients by the envelope theorem: at a solution rho* of
eq. rhoEquation dOmega/drho = 0, so the total derivative of Omega*(V, rho_bath) equals the
explicit partial at rho* (checked with re-solved equilibria, an independent computation)."""
import numpy as np
import pytest

from oracle import functional as F, picard
from paper_0910_1531_gb300 import workloads

SHAPE, H = (8, 8, 8), 0.1
RADIUS, Z = [0.095, 0.181], [1.0, -1.0]


def _setup(molar):
    prob = F.Problem(SHAPE, H, RADIUS, Z, molar)
    V = np.stack([zi * workloads.gaussian_random_field(SHAPE, (H, H, H), 0.3, 0.5, 7) for zi in Z])
    return prob, V


def _solve(prob, V, rho0=None):
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], V.shape).copy() if rho0 is None else rho0.copy()
    rho, it, r = picard.solve(prob, rho, V, tol=1e-13, max_it=2000)
    assert r < 1e-13
    return rho


def test_dOmega_dV_envelope():
    prob, V = _setup([0.5, 0.5])
    rho = _solve(prob, V)
    for (i, zz, yy, xx) in [(0, 1, 2, 3), (1, 5, 0, 6)]:
        d = 1e-4
        vals = []
        for t in (+1, -1):
            Vp = V.copy()
            Vp[i, zz, yy, xx] += t * d
            vals.append(F.grand_potential(prob, _solve(prob, Vp, rho), Vp))
        fd = (vals[0] - vals[1]) / (2 * d)
        assert fd == pytest.approx(F.grad_omega_v(prob, rho)[i, zz, yy, xx], rel=1e-6)


def test_dOmega_dbulk_envelope():
    molar = np.array([0.5, 0.5])
    prob, V = _setup(molar)
    rho = _solve(prob, V)
    partial = F.grad_omega_bulk(SHAPE, H, RADIUS, Z, molar, rho, V)
    for k in range(2):
        step = 1e-3 * molar[k]
        vals = []
        for t in (+1, -1):
            c = molar.copy()
            c[k] += t * step
            pk = F.Problem(SHAPE, H, RADIUS, Z, c)
            vals.append(F.grand_potential(pk, _solve(pk, V, rho), V))
        total = (vals[0] - vals[1]) / (2 * step) / 0.602214076
        assert total == pytest.approx(partial[k], rel=1e-5)
