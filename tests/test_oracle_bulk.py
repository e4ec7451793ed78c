"""Pins of the bath thermodynamics (App. A) against textbook closed forms and limits."""
import math

import numpy as np
import pytest

from oracle.bulk import hs_bath, msa_gamma, msa_mu, make_bath
from oracle.units import bjerrum_length_nm, molar_to_per_nm3


def test_bjerrum_length_water():
    # lambda_B of water at 25 C is ~0.714 nm for eps_r = 78.5 (textbook value).
    assert abs(bjerrum_length_nm(298.15, 78.5) - 0.714) < 1e-3


def test_molar_conversion():
    assert molar_to_per_nm3(1.0) == pytest.approx(0.602214076, rel=1e-15)


@pytest.mark.parametrize("eta", [1e-5, 0.1, 0.25, 0.4])
def test_single_component_percus_yevick(eta):
    # One-component PY compressibility (scaled-particle) closed forms:
    # beta P / rho = (1 + eta + eta^2) / (1 - eta)^3,
    # beta mu_ex = -ln(1 - eta) + eta (14 - 13 eta + 5 eta^2) / (2 (1 - eta)^3).
    R = 0.1
    rho = eta / (4.0 / 3.0 * math.pi * R ** 3)
    mu, bp = hs_bath([rho], [R])
    assert bp / rho == pytest.approx((1 + eta + eta ** 2) / (1 - eta) ** 3, rel=1e-13)
    mu_py = -math.log(1 - eta) + eta * (14 - 13 * eta + 5 * eta ** 2) / (2 * (1 - eta) ** 3)
    assert mu[0] == pytest.approx(mu_py, rel=1e-12, abs=1e-15)


def test_mixture_reduces_to_single_component():
    # Splitting one species into two identical halves changes nothing.
    mu1, p1 = hs_bath([0.6], [0.15])
    mu2, p2 = hs_bath([0.2, 0.4], [0.15, 0.15])
    assert p2 == pytest.approx(p1, rel=1e-14)
    assert np.allclose(mu2, mu1[0], rtol=1e-14)


@pytest.mark.parametrize("c", [0.01, 0.1, 1.0, 2.0])
def test_rpm_gamma_closed_form(c):
    # Restricted primitive model (equal diameters, z = +-1): eta = 0 and
    # 2 sigma Gamma = sqrt(1 + 2 kappa sigma) - 1;  beta mu_ES = -lambda_B Gamma z^2 / (1 + Gamma sigma).
    lb = bjerrum_length_nm(298.15, 78.5)
    R = 0.15
    sigma = 2 * R
    rho = molar_to_per_nm3(c)
    kappa = math.sqrt(4 * math.pi * lb * 2 * rho)
    g_exact = (math.sqrt(1 + 2 * kappa * sigma) - 1) / (2 * sigma)
    g = msa_gamma([rho, rho], [R, R], [1, -1], lb)
    assert g == pytest.approx(g_exact, rel=1e-13)
    mu = msa_mu([rho, rho], [R, R], [1, -1], lb)
    assert np.allclose(mu, -lb * g_exact / (1 + g_exact * sigma), rtol=1e-12)


def test_rpm_divalent_size_symmetric():
    # 2:1 electrolyte of equal sizes: electroneutrality makes eta = 0 again, and
    # Gamma solves 2 Gamma (1 + Gamma sigma) = kappa.
    lb = bjerrum_length_nm(298.15, 78.5)
    R = 0.1
    sigma = 2 * R
    rho = np.array([molar_to_per_nm3(0.05), molar_to_per_nm3(0.1)])
    z = np.array([2.0, -1.0])
    kappa = math.sqrt(4 * math.pi * lb * np.sum(rho * z * z))
    g_exact = (math.sqrt(1 + 2 * kappa * sigma) - 1) / (2 * sigma)
    assert msa_gamma(rho, [R, R], z, lb) == pytest.approx(g_exact, rel=1e-13)


def test_debye_huckel_limit():
    # Gamma -> kappa / 2 and beta mu_ES_i -> -lambda_B z_i^2 kappa / 2 as c -> 0, any sizes.
    lb = bjerrum_length_nm(298.15, 78.5)
    R = [0.095, 0.099, 0.181]
    z = np.array([1.0, 2.0, -1.0])
    c = np.array([1e-9, 1e-10, 1.2e-9])
    rho = np.array([molar_to_per_nm3(v) for v in c])
    kappa = math.sqrt(4 * math.pi * lb * np.sum(rho * z * z))
    g = msa_gamma(rho, R, z, lb)
    assert g == pytest.approx(kappa / 2, rel=1e-4)
    mu = msa_mu(rho, R, z, lb)
    assert np.allclose(mu, -lb * z * z * kappa / 2, rtol=1e-4)


def test_gamma_decreases_screening_below_debye():
    # MSA screening is weaker than Debye at finite size: Gamma < kappa / 2.
    lb = bjerrum_length_nm(298.15, 78.5)
    bath = make_bath([molar_to_per_nm3(0.1)] * 2, [0.095, 0.181], [1, -1], lb)
    kappa = math.sqrt(4 * math.pi * lb * np.sum(bath.rho * bath.z ** 2))
    assert 0 < bath.gamma < kappa / 2
    assert np.all(bath.lam == pytest.approx(bath.radius + 0.5 / bath.gamma))


# ---------------------------------------------------------------------------------------------
# The MSA branch for ions of unequal size (eta != 0).  App. A prints the Gamma equation with its
# auxiliary eta and Omega, and mu^ES, but not the free energy they come from.  The MSA excess
# Helmholtz free energy of the unrestricted primitive model is known independently (Blum's
# internal energy plus Gamma^3 / (3 pi), the Hoye-Blum energy-route result):
#   beta A / V = -lambda_B [Gamma sum_i rho_i z_i^2 / (1 + Gamma sigma_i) + (pi / (2 Delta)) Omega P_n^2]
#                + Gamma^3 / (3 pi),
#   P_n = (1 / Omega) sum_k rho_k sigma_k z_k / (1 + Gamma sigma_k),
#   Omega = 1 + (pi / (2 Delta)) sum_k rho_k sigma_k^3 / (1 + Gamma sigma_k).
# Two facts of that theory pin every term of the oracle's branch: the MSA Gamma is the stationary
# point of beta A / V in Gamma, and the electrostatic chemical potential is its density derivative
# (at the stationary Gamma the total and the fixed-Gamma derivatives coincide).  Derivatives are
# taken by the complex step (no cancellation), which this rational function of Gamma and rho allows.
# ---------------------------------------------------------------------------------------------

def _msa_free_energy(rho, sigma, z, lb, gamma):
    """beta A^MSA / V (kT nm^-3) at a trial Gamma; complex arguments allowed (complex step)."""
    delta = 1.0 - math.pi / 6.0 * np.sum(rho * sigma ** 3)
    den = 1.0 + gamma * sigma
    omega = 1.0 + math.pi / (2.0 * delta) * np.sum(rho * sigma ** 3 / den)
    p_n = np.sum(rho * sigma * z / den) / omega
    energy = -lb * (gamma * np.sum(rho * z * z / den) + math.pi / (2.0 * delta) * omega * p_n ** 2)
    return energy + gamma ** 3 / (3.0 * math.pi)


# (radii nm, valences, molar): the precision and large configurations' baths, the paper's 1 M
# wall electrolyte (R 0.1 / 0.2125 nm) and strongly size-asymmetric 2:1 and 3:1 baths, where
# eta and Omega - 1 are large enough that a slip in either moves Gamma and mu^ES measurably.
_ASYMMETRIC_BATHS = [
    ([0.095, 0.099, 0.181], [1.0, 2.0, -1.0], [0.1, 0.01, 0.12]),
    ([0.095, 0.099, 0.181], [1.0, 2.0, -1.0], [0.1, 0.001, 0.102]),
    ([0.1, 0.2125], [1.0, -1.0], [1.0, 1.0]),
    ([0.1, 0.3], [2.0, -1.0], [1.0, 2.0]),
    ([0.35, 0.09], [3.0, -1.0], [0.5, 1.5]),
]


def _bath_arrays(radii, z, molar):
    return (np.array([molar_to_per_nm3(c) for c in molar]), 2.0 * np.array(radii, dtype=np.float64),
            np.array(z, dtype=np.float64))


@pytest.mark.parametrize("radii,z,molar", _ASYMMETRIC_BATHS)
def test_msa_gamma_is_the_stationary_point_of_the_msa_free_energy(radii, z, molar):
    lb = bjerrum_length_nm(298.15, 78.5)
    rho, sigma, zz = _bath_arrays(radii, z, molar)
    g = msa_gamma(rho, radii, zz, lb)
    step = 1e-30
    dfdg = _msa_free_energy(rho, sigma, zz, lb, g + 1j * step).imag / step
    # the two halves of dA/dGamma (Gamma^2 / pi and the energy part) cancel at the root
    assert abs(dfdg) < 1e-12 * g * g / math.pi, (dfdg, g)
    # and the root is not trivial: eta differs from 0 in every one of these baths
    delta = 1.0 - math.pi / 6.0 * np.sum(rho * sigma ** 3)
    omega = 1.0 + math.pi / (2 * delta) * np.sum(rho * sigma ** 3 / (1 + g * sigma))
    eta = math.pi / (2 * delta * omega) * np.sum(rho * sigma * zz / (1 + g * sigma))
    assert abs(eta) > 1e-4


@pytest.mark.parametrize("radii,z,molar", _ASYMMETRIC_BATHS)
def test_msa_mu_es_is_the_density_derivative_of_the_msa_free_energy(radii, z, molar):
    lb = bjerrum_length_nm(298.15, 78.5)
    rho, sigma, zz = _bath_arrays(radii, z, molar)
    g = msa_gamma(rho, radii, zz, lb)
    mu = msa_mu(rho, radii, zz, lb)
    step = 1e-30
    for i in range(len(rho)):
        rc = rho.astype(np.complex128)
        rc[i] += 1j * step
        d_fixed_gamma = _msa_free_energy(rc, sigma, zz, lb, g).imag / step
        assert mu[i] == pytest.approx(d_fixed_gamma, rel=1e-12, abs=1e-15), (i, mu[i], d_fixed_gamma)
    # total derivative with Gamma re-solved at each density (Richardson-extrapolated central
    # differences): equal to the fixed-Gamma one because Gamma is stationary
    for i in range(len(rho)):
        def total(hrel):
            hh = hrel * rho[i]
            vals = []
            for sgn in (1.0, -1.0):
                r2 = rho.copy()
                r2[i] += sgn * hh
                vals.append(_msa_free_energy(r2, sigma, zz, lb, msa_gamma(r2, radii, zz, lb)))
            return (vals[0] - vals[1]) / (2 * hh)
        d1, d2 = total(1e-3), total(5e-4)
        d = d2 + (d2 - d1) / 3.0
        assert d == pytest.approx(mu[i], rel=1e-7, abs=1e-9), (i, d, mu[i])


def test_msa_free_energy_debye_huckel_limiting_law():
    # beta A / V -> -kappa^3 / (12 pi) as the salt vanishes, whatever the sizes
    lb = bjerrum_length_nm(298.15, 78.5)
    radii, zz = [0.095, 0.099, 0.181], np.array([1.0, 2.0, -1.0])
    rho = np.array([molar_to_per_nm3(c) for c in (1e-9, 1e-10, 1.2e-9)])
    kappa = math.sqrt(4 * math.pi * lb * np.sum(rho * zz * zz))
    g = msa_gamma(rho, radii, zz, lb)
    f = _msa_free_energy(rho, 2 * np.array(radii), zz, lb, g)
    assert f == pytest.approx(-kappa ** 3 / (12 * math.pi), rel=1e-4)
