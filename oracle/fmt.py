"""Antisymmetrised Rosenfeld free-energy density and its derivatives (test infrastructure only).

eq. Phi, with D = 1 - n3 and xi = |nV2|^2 / n2^2:
    Phi = -n0 ln D + (n1 n2 - nV1 . nV2) / D + n2^3 (1 - xi)^3 / (24 pi D^2)

Sec. "Numerical Stability" and App. C (eq. ratio) bound |nV2| <= n2; the
printed inequality |n2|/|nV2| <= 1 is inverted relative to App. C's proof and
is read as xi <= 1.  The bound is enforced by clamping xi to [0, 1]; where
n2 <= 1e-30 the xi-dependent term is taken as 0 (xi treated as 1).

The paper prints no derivatives; they follow from eq. Phi by differentiation:
    dPhi/dn0  = -ln D
    dPhi/dn1  = n2 / D
    dPhi/dn2  = n1 / D + n2^2 (1 - xi)^2 (1 + xi) / (8 pi D^2)
    dPhi/dn3  = n0 / D + (n1 n2 - nV1 . nV2) / D^2 + n2^3 (1 - xi)^3 / (12 pi D^3)
    dPhi/dnV1 = -nV2 / D
    dPhi/dnV2 = -nV1 / D - n2 (1 - xi)^2 nV2 / (4 pi D^2)

Parity: pinned by tests/test_oracle_fmt.py (central finite differences of Phi,
and the uniform-fluid limit, which must reproduce the Percus-Yevick bath
chemical potential and pressure of App. A).
"""

import math

import numpy as np

N2_FLOOR = 1e-30


def _xi(n2, nV2):
    q = nV2[0] ** 2 + nV2[1] ** 2 + nV2[2] ** 2
    safe = n2 > N2_FLOOR
    xi = np.where(safe, q / np.where(safe, n2 * n2, 1.0), 1.0)
    return np.clip(xi, 0.0, 1.0)


def phi(n0, n1, n2, n3, nV1, nV2):
    """Free-energy density Phi (kT / nm^3) of eq. Phi."""
    d = 1.0 - n3
    xi = _xi(n2, nV2)
    dot = nV1[0] * nV2[0] + nV1[1] * nV2[1] + nV1[2] * nV2[2]
    return (-n0 * np.log(d) + (n1 * n2 - dot) / d
            + n2 ** 3 * (1.0 - xi) ** 3 / (24.0 * math.pi * d * d))


def phi_derivatives(n0, n1, n2, n3, nV1, nV2):
    """Return (d0, d1, d2, d3, dV1[3], dV2[3]), the partial derivatives of Phi."""
    d = 1.0 - n3
    xi = _xi(n2, nV2)
    dot = nV1[0] * nV2[0] + nV1[1] * nV2[1] + nV1[2] * nV2[2]
    om = 1.0 - xi
    d0 = -np.log(d)
    d1 = n2 / d
    d2 = n1 / d + n2 * n2 * om * om * (1.0 + xi) / (8.0 * math.pi * d * d)
    d3 = n0 / d + (n1 * n2 - dot) / (d * d) + n2 ** 3 * om ** 3 / (12.0 * math.pi * d ** 3)
    dV1 = [-v / d for v in nV2]
    dV2 = [-nV1[c] / d - n2 * om * om * nV2[c] / (4.0 * math.pi * d * d) for c in range(3)]
    return d0, d1, d2, d3, dV1, dV2
