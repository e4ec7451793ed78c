"""Picard iteration with quadratic line search (test infrastructure only).

Sec. "Nonlinear solver": rho^(1) = G(rho^(0)) (eq. picard); the next iterate
mixes rho^(1) and rho^(0) with a line-search parameter chosen from a quadratic
fit of the squared residual norms sampled along the segment; n3 is bounded by
0.9, which caps the parameter because n3 is linear in rho.

Readings (the paper is ambiguous or silent on these):
* The paper writes rho* = (1 - alpha) rho^(1) + alpha rho^(0) and then bounds
  alpha as the weight of rho^(1).  Here alpha is the weight of the new iterate:
  rho(alpha) = (1 - alpha) rho^(0) + alpha rho^(1); "mixing 0.1" means alpha = 0.1.
* Residual norm: r(rho)^2 = (1/(S N)) sum_i sum_x ((rho_i - G_i) / rho_bath_i)^2,
  the squared L2 norm with each species scaled by its bath density (so that a
  0.001 M species is not invisible next to a 0.1 M one); a fixed-number species
  is scaled by its mean density N_i / (N h^3).
* Samples: r^2 at alpha in {0, alpha_s/2, alpha_s}, alpha_s = min(alpha_max,
  2 alpha_prev) with alpha_prev the previous iteration's alpha (alpha_s =
  alpha_max on the first iteration); the parabola through the three points is
  minimised: if its curvature is positive the vertex, clamped to
  [1e-3 alpha_s, alpha_s], is taken, otherwise the better of the two non-zero
  samples.  (With samples fixed at alpha_max/2 and alpha_max the fit overshoots
  wherever the residual grows much faster than quadratically along the segment,
  e.g. 0.87 M NaCl around a 0.95 nm sphere in a 9.6 nm box, and the iteration
  diverges; tying the interval to the last accepted step keeps the samples on
  the scale where the quadratic model holds.)
* n3 bound, as printed: with M_a = max_x n3(rho^(a))(x),
  alpha_max = min(1, (0.9 - M_0) / (M_1 - M_0)) when M_1 > M_0, else 1.
  (The L-infinity norm is read as the maximum of n3, the packing fraction.)
* Fixed mixing (no line search): alpha = min(mixing, alpha_max).

Parity: solver trajectories are compared, not pinned; the fixed point is
pinned by tests/test_oracle_picard.py (G(rho) = rho at convergence, planar
homogeneity near a wall, Sec. "Verification").  The line-search arithmetic
itself is pinned on a quadratic with a known minimiser.
"""

import math

import numpy as np

from .functional import picard_map, weighted_densities

N3_BOUND = 0.9
ALPHA_FLOOR = 1e-3


def residual_sq(prob, rho, g):
    rb = prob.rho_ref[:, None, None, None]
    return float(np.sum(((rho - g) / rb) ** 2)) / (prob.nspecies * prob.npoints)


def n3_max(prob, rho):
    return float(np.max(weighted_densities(prob, rho)[3]))


def alpha_bound(m0, m1, bound=N3_BOUND):
    if m1 <= m0:
        return 1.0
    return min(1.0, (bound - m0) / (m1 - m0))


def quadratic_alpha(f0, f1, f2, alpha_max):
    """Minimiser of the parabola through (0, f0), (a, f1), (2a, f2), a = alpha_max / 2
    (alpha_max here is the sampled interval alpha_s)."""
    a = 0.5 * alpha_max
    c2 = (f0 - 2.0 * f1 + f2) / (2.0 * a * a)
    c1 = (-3.0 * f0 + 4.0 * f1 - f2) / (2.0 * a)
    if c2 > 0.0:
        vertex = -c1 / (2.0 * c2)
        return min(max(vertex, ALPHA_FLOOR * alpha_max), alpha_max)
    return a if f1 <= f2 else alpha_max


def picard_step(prob, rho0, V, g0=None, mixing=None, alpha_prev=None):
    """One Picard iteration from rho0.  Returns (rho_new, info dict); info["alpha"] is the
    alpha_prev of the next iteration."""
    if g0 is None:
        g0 = picard_map(prob, rho0, V)
    rho1 = g0
    f0 = residual_sq(prob, rho0, rho1)
    alpha_max = alpha_bound(n3_max(prob, rho0), n3_max(prob, rho1))
    info = {"resid": math.sqrt(f0), "alpha_max": alpha_max}
    if mixing is not None:
        alpha = min(mixing, alpha_max)
    else:
        alpha_s = alpha_max if alpha_prev is None else min(alpha_max, 2.0 * alpha_prev)
        samples = []
        for t in (0.5 * alpha_s, alpha_s):
            rt = (1.0 - t) * rho0 + t * rho1
            samples.append(residual_sq(prob, rt, picard_map(prob, rt, V)))
        info["f"] = (f0, samples[0], samples[1])
        info["alpha_s"] = alpha_s
        alpha = quadratic_alpha(f0, samples[0], samples[1], alpha_s)
    info["alpha"] = alpha
    return (1.0 - alpha) * rho0 + alpha * rho1, info


def solve(prob, rho, V, tol, max_it, mixing=None):
    """Iterate until r(rho) < tol or max_it iterations; returns (rho, iterations, r)."""
    g = picard_map(prob, rho, V)
    r = math.sqrt(residual_sq(prob, rho, g))
    it = 0
    alpha_prev = None
    while it < max_it and r >= tol:
        rho, info = picard_step(prob, rho, V, g0=g, mixing=mixing, alpha_prev=alpha_prev)
        alpha_prev = info["alpha"]
        g = picard_map(prob, rho, V)
        r = math.sqrt(residual_sq(prob, rho, g))
        it += 1
    return rho, it, r
