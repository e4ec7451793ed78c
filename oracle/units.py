"""Physical constants and unit conversions (test infrastructure only).

Units used throughout the oracle: lengths in nm, energies in kT, number
densities in nm^-3.  The paper writes the Poisson equation (eq. Poisson) with a
dielectric coefficient epsilon; it is read as eps0 * eps_r everywhere (the
paper mixes "epsilon" and "epsilon epsilon_0" between eq. Gamma and the MSA
bath potential of App. A).  With that reading e^2 / (4 pi eps0 eps_r kT) is the
Bjerrum length lambda_B, and the reduced potential psi = e phi / kT obeys
-Laplace(psi) = 4 pi lambda_B sum_i z_i rho_i.

Parity: pinned by tests/test_oracle_bulk.py (lambda_B at 298.15 K, eps_r 78.5).
"""

import math

E_CHARGE = 1.602176634e-19      # C, exact (SI 2019)
K_BOLTZMANN = 1.380649e-23      # J/K, exact (SI 2019)
N_AVOGADRO = 6.02214076e23      # 1/mol, exact (SI 2019)
EPS0 = 8.8541878128e-12         # F/m, CODATA 2018


def bjerrum_length_nm(temperature_K: float, eps_r: float) -> float:
    """lambda_B = e^2 / (4 pi eps0 eps_r k T), in nm."""
    return E_CHARGE ** 2 / (4.0 * math.pi * EPS0 * eps_r * K_BOLTZMANN * temperature_K) * 1e9


def molar_to_per_nm3(c_molar: float) -> float:
    """mol/L -> particles per nm^3 (1 L = 1e24 nm^3)."""
    return c_molar * N_AVOGADRO * 1e-24
