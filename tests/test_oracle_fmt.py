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


# ---- the other hard-sphere forms (Rosenfeld 1989, White Bear 2002) ----------------------------

@pytest.mark.parametrize("kind", ["rosenfeld", "white_bear"])
def test_other_forms_derivatives_match_central_differences(kind):
    rng = np.random.default_rng(6)
    state = _random_state(rng)
    state[3] = np.concatenate([rng.uniform(1e-4, 0.05, 10), rng.uniform(0.05, 0.85, 30)])   # both WB branches
    v = _flat(state)
    d = fmt.phi_derivatives(*_unflat(v), kind=kind)
    dflat = np.concatenate([[d[0], d[1], d[2], d[3]], d[4], d[5]])
    for a in range(10):
        eps = 3e-4 * np.maximum(np.abs(v[a]), 0.1)
        if a == 3:
            eps = np.minimum(eps, 0.2 * v[3])

        def at(t):
            w = v.copy()
            w[a] = w[a] + t * eps
            return fmt.phi(*_unflat(w), kind=kind)
        fd = (-at(2) + 8 * at(1) - 8 * at(-1) + at(-2)) / (12 * eps)
        assert np.allclose(dflat[a], fd, rtol=1e-7, atol=1e-8), (kind, a)


def test_rosenfeld_form_equals_eq_phi_without_vectors_and_white_bear_tends_to_it():
    # With n_V = 0 the original Rosenfeld form is eq. Phi; White Bear's f(n3) -> 1/(24 pi) as n3 -> 0.
    rng = np.random.default_rng(7)
    n0, n1, n2, n3, _, _ = _random_state(rng)
    zero = [0.0, 0.0, 0.0]
    assert np.allclose(fmt.phi(n0, n1, n2, n3, zero, zero, kind="rosenfeld"), fmt.phi(n0, n1, n2, n3, zero, zero),
                       rtol=1e-14)
    f, _ = fmt._tensor_f(np.array([1e-9]), "white_bear")
    assert f[0] == pytest.approx(1.0 / (24.0 * math.pi), rel=1e-8)


def test_white_bear_series_matches_closed_form():
    # Below n3 = 0.5 g(n3) = (n3 + D^2 ln D)/n3^2 is summed as a series; compare with the closed form
    # where the closed form keeps its digits (n3 >= 0.05) and with high-precision values at small n3.
    n3 = np.linspace(0.05, 0.499, 50)
    g, dg = fmt._wb_g(n3)
    d = 1.0 - n3
    ln_d = np.log(d)
    num = n3 + d * d * ln_d
    assert np.allclose(g, num / n3 ** 2, rtol=1e-12)
    assert np.allclose(dg, (n3 - 2 * d * ln_d) / n3 ** 2 - 2 * num / n3 ** 3, rtol=1e-9)
    import decimal
    decimal.getcontext().prec = 60
    for t in ("1e-6", "0.001", "0.02"):
        x = decimal.Decimal(t)
        dd = 1 - x
        exact = (x + dd * dd * dd.ln()) / (x * x)
        assert float(fmt._wb_g(np.array([float(x)]))[0][0]) == pytest.approx(float(exact), rel=1e-14)


@pytest.mark.parametrize("eta", [1e-5, 0.1, 0.25, 0.4])
def test_white_bear_uniform_limit_is_carnahan_starling(eta):
    # One component: beta mu_ex = (8 eta - 9 eta^2 + 3 eta^3)/(1 - eta)^3 and
    # beta P / rho = (1 + eta + eta^2 - eta^3)/(1 - eta)^3 (Carnahan-Starling).
    from oracle.bulk import hs_bath_fmt
    R = 0.1
    rho = eta / (4.0 / 3.0 * math.pi * R ** 3)
    mu, p = hs_bath_fmt([rho], [R], "white_bear")
    e = eta
    assert mu[0] == pytest.approx((8 * e - 9 * e ** 2 + 3 * e ** 3) / (1 - e) ** 3, rel=1e-12, abs=1e-15)
    assert p == pytest.approx(rho * (1 + e + e ** 2 - e ** 3) / (1 - e) ** 3, rel=1e-12)


@pytest.mark.parametrize("rho,R", [
    ([0.602, 0.602], [0.1, 0.2125]),
    ([3.0, 1.0, 0.5], [0.1, 0.15, 0.2]),
])
def test_white_bear_uniform_mixture_pressure_is_bmcsl(rho, R):
    # Mixture: beta P = (6/pi) [xi0/D + 3 xi1 xi2/D^2 + (3 - xi3) xi2^3/D^3] (BMCSL), xi_n = (pi/6)
    # sum rho sigma^n; the chemical potentials obey Gibbs-Duhem with it (dP = sum rho_i dmu_i).
    from oracle.bulk import hs_bath_fmt
    rho, R = np.asarray(rho), np.asarray(R)
    sig = 2 * R
    xi = [math.pi / 6 * np.sum(rho * sig ** n) for n in range(4)]
    D = 1 - xi[3]
    p_bmcsl = 6 / math.pi * (xi[0] / D + 3 * xi[1] * xi[2] / D ** 2 + (3 - xi[3]) * xi[2] ** 3 / D ** 3)
    mu, p = hs_bath_fmt(rho, R, "white_bear")
    assert p == pytest.approx(p_bmcsl, rel=1e-12)
    for k in range(len(rho)):
        h = 1e-5 * rho[k]
        rp, rm = rho.copy(), rho.copy()
        rp[k] += h
        rm[k] -= h
        mp, pp = hs_bath_fmt(rp, R, "white_bear")
        mm, pm = hs_bath_fmt(rm, R, "white_bear")
        # ideal part: d(sum rho)/drho_k = 1 plus sum_i rho_i dmu_ex_i/drho_k
        lhs = (pp - pm) / (2 * h)
        rhs = 1.0 + np.sum(rho * (mp - mm) / (2 * h))
        assert lhs == pytest.approx(rhs, rel=1e-7)
