"""Pins of eq. Phi and its derivatives: finite differences, the |nV2| <= n2 clamp,
and the uniform-fluid limit, which must give App. A's Percus-Yevick bath values."""
import math

import numpy as np
import pytest

from oracle import fmt
from oracle.bulk import hs_bath


def _random_state(rng, m=40):
    n3 = rng.uniform(0.01, 0.85, m)
    n2 = rng.uniform(0.5, 8.0, m)
    n1 = rng.uniform(0.05, 1.0, m)
    n0 = rng.uniform(0.1, 5.0, m)
    direction = rng.standard_normal((3, m))
    direction /= np.linalg.norm(direction, axis=0)
    nV2 = direction * n2 * rng.uniform(0.0, 0.95, m)
    nV1 = rng.standard_normal((3, m)) * 0.2
    return [n0, n1, n2, n3, nV1, nV2]


def _flat(state):
    n0, n1, n2, n3, nV1, nV2 = state
    return np.concatenate([[n0, n1, n2, n3], nV1, nV2])


def _unflat(v):
    return [v[0], v[1], v[2], v[3], [v[4], v[5], v[6]], [v[7], v[8], v[9]]]


def test_derivatives_match_central_differences():
    rng = np.random.default_rng(5)
    v = _flat(_random_state(rng))
    d = fmt.phi_derivatives(*_unflat(v))
    dflat = np.concatenate([[d[0], d[1], d[2], d[3]], d[4], d[5]])
    for a in range(10):
        eps = 3e-4 * np.maximum(np.abs(v[a]), 0.1)

        def at(t):
            w = v.copy()
            w[a] = w[a] + t * eps
            return fmt.phi(*_unflat(w))
        fd = (-at(2) + 8 * at(1) - 8 * at(-1) + at(-2)) / (12 * eps)   # fourth-order stencil
        assert np.allclose(dflat[a], fd, rtol=1e-8, atol=1e-8), a


def test_clamp_beyond_bound_equals_bound():
    # xi > 1 (|nV2| > n2, Sec. "Numerical Stability") contributes like xi = 1: the n2^3 term vanishes.
    n0, n1, n2, n3 = 1.0, 0.3, 2.0, 0.3
    nV1 = [0.0, 0.0, 0.1]
    over = fmt.phi(n0, n1, n2, n3, nV1, [0.0, 0.0, 2.5])
    plain = -n0 * math.log(1 - n3) + (n1 * n2 - 0.1 * 2.5) / (1 - n3)
    assert over == pytest.approx(plain, rel=1e-15)
    d = fmt.phi_derivatives(n0, n1, n2, n3, nV1, [0.0, 0.0, 2.5])
    assert d[2] == pytest.approx(n1 / (1 - n3))
    assert d[5][2] == pytest.approx(-0.1 / (1 - n3))


def _uniform_measures(rho, R):
    rho, R = np.asarray(rho), np.asarray(R)
    return (np.sum(rho), np.sum(rho * R), np.sum(rho * 4 * math.pi * R ** 2),
            np.sum(rho * 4 * math.pi * R ** 3 / 3))


@pytest.mark.parametrize("rho,R", [
    ([0.0602, 0.0602], [0.095, 0.181]),
    ([0.0602, 0.00602, 0.0723], [0.095, 0.099, 0.181]),
    ([0.4 / (4 / 3 * math.pi * 0.1 ** 3)], [0.1]),
    ([3.0, 1.0, 0.5], [0.1, 0.15, 0.2]),
])
def test_uniform_limit_is_percus_yevick(rho, R):
    # For constant densities n_alpha are the fundamental measures (Sec. "Verification"),
    # n_V = 0, and beta mu_HS_i = sum_alpha dPhi/dn_alpha w_hat_i^alpha(0) must equal
    # eq. muHSBath; beta P = sum rho + sum rho mu - Phi must equal eq. HSPressure.
    n0, n1, n2, n3 = _uniform_measures(rho, R)
    zero = [0.0, 0.0, 0.0]
    d0, d1, d2, d3, _, _ = fmt.phi_derivatives(n0, n1, n2, n3, zero, zero)
    R = np.asarray(R)
    mu = d0 + d1 * R + d2 * 4 * math.pi * R ** 2 + d3 * 4 * math.pi * R ** 3 / 3
    mu_py, p_py = hs_bath(rho, R)
    assert np.allclose(mu, mu_py, rtol=1e-13)
    p = np.sum(rho) + np.sum(np.asarray(rho) * mu) - fmt.phi(n0, n1, n2, n3, zero, zero)
    assert p == pytest.approx(p_py, rel=1e-13)
