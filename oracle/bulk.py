"""Bath (bulk) thermodynamics, App. A (test infrastructure only).

* Percus-Yevick / scaled-particle hard-sphere bath chemical potential
  (eq. muHSBath) and pressure (eq. HSPressure), with sigma_i = 2 R_i; for the White Bear
  functional (an alternative Phi_HS, see fmt.py) the uniform limit of that functional instead.
* MSA screening parameter Gamma from the implicit equation eq. Gamma, with the
  auxiliary eta and Omega printed beneath it, and the electrostatic bath
  chemical potential mu^{ES,bath} printed last in App. A.

All quantities in kT units, lengths in nm, densities in nm^-3.
eq. Gamma reads 4 Gamma^2 = e^2/(kT eps) sum_j rho_j ((z_j - eta sigma_j^2) /
(1 + Gamma sigma_j))^2; with eps = eps0 eps_r, e^2/(kT eps) = 4 pi lambda_B, so
Gamma^2 = pi lambda_B sum_j (...)^2.  Gamma is found by plain bisection on
[0, kappa] (kappa the Debye parameter): slow, but its convergence needs no
argument beyond continuity and a sign change.

Parity: pinned (tests/test_oracle_bulk.py) by the textbook single-component
Percus-Yevick compressibility pressure and chemical potential, the closed-form
restricted-primitive-model Gamma, the Debye-Hueckel limit, and (in
tests/test_oracle_fmt.py) by the bulk limit of the FMT functional eq. Phi.  The
size-asymmetric MSA branch (eta != 0: eta, Omega, the eta terms of eq. Gamma and of
mu^ES) is pinned by the MSA free energy of the unrestricted primitive model (Blum's
internal energy plus Gamma^3 / (3 pi)), which App. A does not print: Gamma must be its
stationary point and mu^ES its density derivative, on baths with eta up to O(0.1).
"""

import math
from dataclasses import dataclass

import numpy as np


def hs_bath(rho, radius):
    """Return (beta mu^HS_i array, beta P^HS) from eqs. muHSBath and HSPressure."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = 2.0 * np.asarray(radius, dtype=np.float64)
    xi = [math.pi / 6.0 * float(np.sum(rho * sigma ** n)) for n in range(4)]
    delta = 1.0 - xi[3]
    beta_p = 6.0 / math.pi * (xi[0] / delta + 3.0 * xi[1] * xi[2] / delta ** 2
                              + 3.0 * xi[2] ** 3 / delta ** 3)
    mu = (-math.log(delta)
          + (3.0 * xi[2] * sigma + 3.0 * xi[1] * sigma ** 2) / delta
          + 9.0 * xi[2] ** 2 * sigma ** 2 / (2.0 * delta ** 2)
          + math.pi * beta_p * sigma ** 3 / 6.0)
    return mu, beta_p


def _msa_eta_omega(gamma, rho, sigma, z, delta):
    """eta and Omega of App. A at a trial Gamma."""
    omega = 1.0 + math.pi / (2.0 * delta) * float(np.sum(rho * sigma ** 3 / (1.0 + gamma * sigma)))
    eta = math.pi / (2.0 * delta * omega) * float(np.sum(rho * sigma * z / (1.0 + gamma * sigma)))
    return eta, omega


def _gamma_equation(gamma, rho, sigma, z, delta, lb):
    """Gamma^2 - pi lambda_B sum_j rho_j ((z_j - eta sigma_j^2)/(1 + Gamma sigma_j))^2."""
    eta, _ = _msa_eta_omega(gamma, rho, sigma, z, delta)
    rhs = math.pi * lb * float(np.sum(rho * ((z - eta * sigma ** 2) / (1.0 + gamma * sigma)) ** 2))
    return gamma * gamma - rhs


def msa_gamma(rho, radius, z, lb):
    """MSA Gamma (nm^-1) solving eq. Gamma, by bisection on [0, kappa]."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = 2.0 * np.asarray(radius, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    delta = 1.0 - math.pi / 6.0 * float(np.sum(rho * sigma ** 3))
    kappa = math.sqrt(4.0 * math.pi * lb * float(np.sum(rho * z * z)))
    if kappa == 0.0:
        return 0.0
    lo, hi = 0.0, kappa
    f_lo = _gamma_equation(lo, rho, sigma, z, delta, lb)
    f_hi = _gamma_equation(hi, rho, sigma, z, delta, lb)
    while f_hi <= 0.0:          # widen until the sign changes (never needed in practice)
        hi *= 2.0
        f_hi = _gamma_equation(hi, rho, sigma, z, delta, lb)
    assert f_lo < 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        f_mid = _gamma_equation(mid, rho, sigma, z, delta, lb)
        if f_mid < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def msa_mu(rho, radius, z, lb, gamma=None):
    """beta mu^{ES,bath}_i (App. A, last equation), eps read as eps0 eps_r."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = 2.0 * np.asarray(radius, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    if gamma is None:
        gamma = msa_gamma(rho, radius, z, lb)
    delta = 1.0 - math.pi / 6.0 * float(np.sum(rho * sigma ** 3))
    eta, _ = _msa_eta_omega(gamma, rho, sigma, z, delta)
    return -lb * (gamma * z * z / (1.0 + gamma * sigma)
                  + eta * sigma * ((2.0 * z - eta * sigma ** 2) / (1.0 + gamma * sigma)
                                   + eta * sigma ** 2 / 3.0))


@dataclass
class Bath:
    """Bath state: densities, chemical potentials and the MSA parameters."""
    rho: np.ndarray          # nm^-3
    radius: np.ndarray       # nm
    z: np.ndarray            # valences
    lb: float                # Bjerrum length, nm
    mu_hs: np.ndarray        # beta mu^{HS,bath}
    beta_p: float            # beta P^{HS}_bath, nm^-3
    gamma: float             # MSA Gamma, nm^-1
    mu_es: np.ndarray        # beta mu^{ES,bath}
    lam: np.ndarray          # lambda_k = R_k + 1/(2 Gamma) (Sec. "Bulk Fluid Method")

    @property
    def mu_ex(self):
        return self.mu_hs + self.mu_es


def hs_bath_fmt(rho, radius, kind):
    """(beta mu^HS_i, beta P^HS) of a uniform fluid under the FMT form `kind` (fmt.KINDS): with
    n_alpha = sum_j rho_j w_hat_j^alpha(0) (the fundamental measures 1, R, 4 pi R^2, 4 pi R^3/3)
    and n_V = 0, beta mu_i = sum_alpha dPhi/dn_alpha w_hat_i^alpha(0) and beta P = n0 + sum_alpha
    n_alpha dPhi/dn_alpha - Phi.  For rslt and rosenfeld this is App. A's Percus-Yevick bath."""
    from . import fmt
    rho = np.asarray(rho, dtype=np.float64)
    R = np.asarray(radius, dtype=np.float64)
    w = [np.ones_like(R), R, 4.0 * math.pi * R ** 2, 4.0 * math.pi * R ** 3 / 3.0]
    n = [float(np.sum(rho * wa)) for wa in w]
    zero = [0.0, 0.0, 0.0]
    d = fmt.phi_derivatives(n[0], n[1], n[2], n[3], zero, zero, kind)[:4]
    mu = sum(float(d[a]) * w[a] for a in range(4))
    beta_p = n[0] + sum(n[a] * float(d[a]) for a in range(4)) - float(fmt.phi(n[0], n[1], n[2], n[3], zero, zero, kind))
    return mu, beta_p


def make_bath(rho, radius, z, lb, functional="rslt"):
    rho = np.asarray(rho, dtype=np.float64)
    radius = np.asarray(radius, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    if functional == "white_bear":
        mu_hs, beta_p = hs_bath_fmt(rho, radius, functional)
    else:
        mu_hs, beta_p = hs_bath(rho, radius)
    gamma = msa_gamma(rho, radius, z, lb)
    mu_es = msa_mu(rho, radius, z, lb, gamma)
    lam = radius + (0.5 / gamma if gamma > 0.0 else np.inf)
    return Bath(rho=rho, radius=radius, z=z, lb=lb, mu_hs=mu_hs, beta_p=beta_p,
                gamma=gamma, mu_es=mu_es, lam=lam)
