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
