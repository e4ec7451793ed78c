"""Hard-sphere FMT free-energy densities and their derivatives (test infrastructure only).

The paper uses the antisymmetrised Rosenfeld form (eq. Phi, kind "rslt", the default) and notes
that other Phi_HS of the literature it cites leave the numerical scheme unchanged; two of them are
here as well (kind "rosenfeld": the original 1989 form; kind "white_bear": the 2002 White Bear
form), written from their published definitions.

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

Both other forms replace the last term by T(n2, nV2) f(n3), T = n2^3 - 3 n2 nV2 . nV2 (no clamp):
    rosenfeld:  f = 1 / (24 pi D^2)
    white_bear: f = (n3 + D^2 ln D) / (36 pi n3^2 D^2)
so that
    dPhi/dn2  = n1 / D + 3 (n2^2 - nV2 . nV2) f,   dPhi/dn3 = n0 / D + (n1 n2 - nV1 . nV2) / D^2 + T f'
    dPhi/dnV2 = -nV1 / D - 6 n2 nV2 f              (dPhi/dn0, dn1, dnV1 as above).
For white_bear, g = f 36 pi D^2 = (n3 + D^2 ln D) / n3^2 loses its digits to cancellation as
n3 -> 0; below n3 = 0.5 it is summed from its power series, g = 3/2 - sum_{k>=3} 2 n3^(k-2) /
(k (k-1) (k-2)), g' = -sum_{k>=3} 2 n3^(k-3) / (k (k-1)) (the expansion of ln D), and
f' = (g' D + 2 g) / (36 pi D^3).  g(0) = 3/2 gives f(0) = 1/(24 pi), the Rosenfeld value.

Parity: pinned by tests/test_oracle_fmt.py (central finite differences of Phi for every kind,
the uniform-fluid limit, which must reproduce the Percus-Yevick bath chemical potential and
pressure of App. A for rslt and rosenfeld and the Carnahan-Starling / BMCSL ones for white_bear,
and the series against the closed form).
"""

import math

import numpy as np

N2_FLOOR = 1e-30


def _xi(n2, nV2):
    q = nV2[0] ** 2 + nV2[1] ** 2 + nV2[2] ** 2
    safe = n2 > N2_FLOOR
    xi = np.where(safe, q / np.where(safe, n2 * n2, 1.0), 1.0)
    return np.clip(xi, 0.0, 1.0)


KINDS = ("rslt", "rosenfeld", "white_bear")
WB_SERIES_BELOW = 0.5
_WB_TERMS = 60


def _wb_g(n3):
    """g(n3) = (n3 + D^2 ln D) / n3^2 and its derivative (white_bear), D = 1 - n3."""
    n3 = np.asarray(n3, dtype=np.float64)
    small = n3 < WB_SERIES_BELOW
    t = np.where(small, n3, 0.0)
    g_s = np.full_like(t, 1.5)
    dg_s = np.zeros_like(t)
    p = np.ones_like(t)          # t^(k-3)
    for k in range(3, 3 + _WB_TERMS):
        g_s = g_s - 2.0 * p * t / (k * (k - 1) * (k - 2))
        dg_s = dg_s - 2.0 * p / (k * (k - 1))
        p = p * t
    u = np.where(small, 0.5, n3)
    d = 1.0 - u
    ln_d = np.log(d)
    num = u + d * d * ln_d
    g_c = num / (u * u)
    dg_c = (u - 2.0 * d * ln_d) / (u * u) - 2.0 * num / (u ** 3)
    return np.where(small, g_s, g_c), np.where(small, dg_s, dg_c)


def _tensor_f(n3, kind):
    """f(n3) and f'(n3) of the rosenfeld / white_bear forms."""
    d = 1.0 - n3
    if kind == "rosenfeld":
        return 1.0 / (24.0 * math.pi * d * d), 1.0 / (12.0 * math.pi * d ** 3)
    g, dg = _wb_g(n3)
    return g / (36.0 * math.pi * d * d), (dg * d + 2.0 * g) / (36.0 * math.pi * d ** 3)


def phi(n0, n1, n2, n3, nV1, nV2, kind="rslt"):
    """Free-energy density Phi (kT / nm^3): eq. Phi (kind "rslt") or another form of KINDS."""
    if kind != "rslt":
        d = 1.0 - n3
        q = nV2[0] ** 2 + nV2[1] ** 2 + nV2[2] ** 2
        dot = nV1[0] * nV2[0] + nV1[1] * nV2[1] + nV1[2] * nV2[2]
        f, _ = _tensor_f(n3, kind)
        return -n0 * np.log(d) + (n1 * n2 - dot) / d + (n2 ** 3 - 3.0 * n2 * q) * f
    d = 1.0 - n3
    xi = _xi(n2, nV2)
    dot = nV1[0] * nV2[0] + nV1[1] * nV2[1] + nV1[2] * nV2[2]
    return (-n0 * np.log(d) + (n1 * n2 - dot) / d
            + n2 ** 3 * (1.0 - xi) ** 3 / (24.0 * math.pi * d * d))


def phi_derivatives(n0, n1, n2, n3, nV1, nV2, kind="rslt"):
    """Return (d0, d1, d2, d3, dV1[3], dV2[3]), the partial derivatives of Phi."""
    if kind != "rslt":
        d = 1.0 - n3
        q = nV2[0] ** 2 + nV2[1] ** 2 + nV2[2] ** 2
        dot = nV1[0] * nV2[0] + nV1[1] * nV2[1] + nV1[2] * nV2[2]
        f, df = _tensor_f(n3, kind)
        d0 = -np.log(d)
        d1 = n2 / d
        d2 = n1 / d + 3.0 * (n2 * n2 - q) * f
        d3 = n0 / d + (n1 * n2 - dot) / (d * d) + (n2 ** 3 - 3.0 * n2 * q) * df
        dV1 = [-v / d for v in nV2]
        dV2 = [-nV1[c] / d - 6.0 * n2 * nV2[c] * f for c in range(3)]
        return d0, d1, d2, d3, dV1, dV2
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
