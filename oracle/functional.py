"""Weighted densities, back-convolution, electrostatics and the map G (test infrastructure only).

Discretisation (Sec. "Discretization and Solution in Equilibrium"): periodic
grid, convolutions evaluated with the convolution theorem (eq. conv) using the
analytic weight transforms sampled on the DFT wave vectors (App. B).  With
DFT/IDFT as in ``oracle.fourier`` (IDFT carries 1/N), the continuous
convolution integral of a grid field f with a kernel w becomes
IDFT(DFT(f) * w_hat), without a factor h^3, because w_hat is the continuous
transform.

* eq. nDef, n_alpha(x) = sum_i int rho_i(x') w_i(x' - x) dx', is a
  cross-correlation: its transform is rho_hat_i(k) w_hat_i(-k).  The scalar
  weights are even (w_hat(-k) = w_hat(k)); the vector weights are odd
  (w_hat(-k) = -w_hat(k)), which makes n_V2 = +grad n3.
* eq. muHS, mu_HS_i(x) = sum_alpha int dPhi/dn_alpha(x') w_i(x - x') dx', is a
  true convolution: transform Phi_hat_alpha(k) w_hat_i(+k).
* Real fields are recovered as the real part of the complex inverse DFT.  For
  an even N_d this sets the d-component of the vector terms to zero at the
  Nyquist index j_d = N_d/2, where the sampled odd weight is not Hermitian.

Component order of the ten weighted densities everywhere in this project:
    [n0, n1, n2, n3, nV1x, nV1y, nV1z, nV2x, nV2y, nV2z].

Electrostatics:
* eq. potentialSolution / eq. potentialConstraint, in reduced form
  psi = e phi / kT:  psi_hat = 4 pi lambda_B sum_j z_j rho_hat_j / lap(k),
  psi_hat(0) = 0, lap(k) = sum_d 2 (1 - cos(k_d h_d)) / h_d^2.
* eq. muESexpansion:  mu_SC_i = mu_ES_bath_i - sum_j DC_ij (*) (rho_j - rho_bath_j);
  DFT(rho_j - rho_bath_j) = rho_hat_j - N rho_bath_j delta_{k,0} (the
  constant's transform), so only inverse transforms are added (Sec. "Bulk Fluid
  Method").

Fixed-point map (eq. rhoEquation with eq. excessChemicalPotential):
    G_i(x) = rho_bath_i exp(mu_ex_bath_i - V_i(x) - mu_HS_i(x) - mu_SC_i(x) - z_i psi(x))
with mu_ex_bath = mu_HS_bath + mu_ES_bath (App. A).  eq. rhoEquation writes
exp((mu_bath - mu_ext - mu_ex)/kT); App. A's mu_bath holds only the excess
parts, so the ideal part kT ln rho_bath is read as the prefactor rho_bath_i.
Voxels with V_i = +inf (hard exclusion) give G_i = 0.

Grand potential (not printed in the paper; the functional whose stationarity
is eq. rhoEquation, with the bulk-fluid expansion eq. muESexpansion read as a
second-order free-energy expansion about the bath):
    Omega/kT = h^3 sum_x sum_i [rho_i (ln(rho_i/rho_bath_i) - 1) + rho_i (V_i - mu_ex_bath_i)]
             + h^3 sum_x Phi(n(x))
             + (h^3/2) sum_x q(x) psi(x),             q = sum_i z_i rho_i
             + h^3 sum_i mu_ES_bath_i sum_x drho_i(x)
             - (h^3/2) sum_ij sum_x drho_i(x) (DC_ij (*) drho_j)(x)
so that dOmega/drho_i(x) = h^3 [ln(rho_i/rho_bath_i) + V_i - mu_ex_bath_i + mu_ex_i(x)],
dOmega/dV_i(x) = h^3 rho_i(x), and dOmega/drho_bath_k follows by differentiating over the bath.

Parity: pinned by tests/test_oracle_functional.py (uniform fluid -> the
fundamental measures, E1/E2 of Sec. "Verification"; a single Fourier mode with
weights from quadrature; n_V2 against finite differences of n3; the FD
Laplacian applied to psi in real space; the uniform bath as a fixed point of G;
finite differences of Omega for its gradient).
"""

import math

import numpy as np

from . import fourier, weights, fmt
from .bulk import make_bath
from .units import bjerrum_length_nm, molar_to_per_nm3

N_COMPONENTS = 10


class Problem:
    """Grid, species and bath of one state point.

    shape = (Nz, Ny, Nx); h = (hx, hy, hz) in nm; radius in nm; z valences;
    bulk_molar in mol/L.
    """

    def __init__(self, shape, h, radius, z, bulk_molar, temperature_K=298.15, eps_r=78.5, n_fixed=None,
                 functional="rslt"):
        self.shape = tuple(int(s) for s in shape)
        if np.isscalar(h):
            h = (h, h, h)
        self.h = tuple(float(v) for v in h)
        self.radius = np.asarray(radius, dtype=np.float64)
        self.z = np.asarray(z, dtype=np.float64)
        self.nspecies = len(self.radius)
        self.lb = bjerrum_length_nm(temperature_K, eps_r)
        rho_b = np.array([molar_to_per_nm3(c) for c in bulk_molar], dtype=np.float64)
        # hard-sphere free-energy density: eq. Phi ("rslt") or another form of fmt.KINDS
        if functional not in fmt.KINDS:
            raise ValueError(f"unknown functional {functional!r}")
        self.functional = functional
        self.bath = make_bath(rho_b, self.radius, self.z, self.lb, functional)
        self.npoints = self.shape[0] * self.shape[1] * self.shape[2]
        self.dv = self.h[0] * self.h[1] * self.h[2]
        # Fixed-number (canonical) species: n_fixed[i] > 0 particles in the box, not in the bath
        # (bulk_molar[i] = 0).  rho_ref: the residual weights (bath density, or the species'
        # mean density N_i / (N h^3) for a fixed-number species).
        self.n_fixed = np.zeros(self.nspecies) if n_fixed is None else np.asarray(n_fixed, dtype=np.float64)
        self.canonical = self.n_fixed > 0.0
        self.rho_ref = np.where(self.canonical, self.n_fixed / (self.npoints * self.dv), self.bath.rho)
        kz, ky, kx = fourier.kgrid(self.shape, self.h)
        self.kvec = (kz, ky, kx)
        self.kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
        self.w = [weights.fmt_weights_hat(kz, ky, kx, R) for R in self.radius]
        self.lap = weights.laplacian_symbol(kz, ky, kx, self.h)
        lam = self.bath.lam
        S = self.nspecies
        self.dc_hat = [[weights.delta_c_hat(self.kmag, self.z[i], self.z[j], lam[i], lam[j],
                                            self.radius[i] + self.radius[j], self.lb)
                        for j in range(S)] for i in range(S)]


def weighted_densities(prob, rho):
    """The ten n_alpha fields (eq. nDef via eq. conv); rho has shape (S, Nz, Ny, Nx)."""
    rho_hat = fourier.dft3(rho)
    acc = [np.zeros(prob.shape, dtype=np.complex128) for _ in range(N_COMPONENTS)]
    for i in range(prob.nspecies):
        w0, w1, w2, w3, wV1, wV2 = prob.w[i]
        r = rho_hat[i]
        acc[0] += r * w0
        acc[1] += r * w1
        acc[2] += r * w2
        acc[3] += r * w3
        for c in range(3):
            acc[4 + c] += r * (-wV1[c])      # w_hat(-k) = -w_hat(k) for odd weights
            acc[7 + c] += r * (-wV2[c])
    return np.real(fourier.idft3(np.stack(acc)))


def phi_derivative_fields(n, kind="rslt"):
    """The ten dPhi/dn_alpha fields for weighted densities n (10, Nz, Ny, Nx)."""
    d0, d1, d2, d3, dV1, dV2 = fmt.phi_derivatives(n[0], n[1], n[2], n[3], n[4:7], n[7:10], kind)
    return np.stack([d0, d1, d2, d3] + list(dV1) + list(dV2))


def phi_field(n, kind="rslt"):
    return fmt.phi(n[0], n[1], n[2], n[3], n[4:7], n[7:10], kind)


def mu_hs(prob, dphi):
    """beta mu_HS_i(x) (eq. muHS via eq. conv) from the ten dPhi/dn_alpha fields."""
    dphi_hat = fourier.dft3(dphi)
    out = []
    for i in range(prob.nspecies):
        w0, w1, w2, w3, wV1, wV2 = prob.w[i]
        acc = dphi_hat[0] * w0 + dphi_hat[1] * w1 + dphi_hat[2] * w2 + dphi_hat[3] * w3
        for c in range(3):
            acc = acc + dphi_hat[4 + c] * wV1[c] + dphi_hat[7 + c] * wV2[c]
        out.append(acc)
    return np.real(fourier.idft3(np.stack(out)))


def psi(prob, rho):
    """Reduced mean-field potential psi = e phi / kT (eq. potentialSolution, psi_hat(0) = 0)."""
    q_hat = fourier.dft3(np.tensordot(prob.z, rho, axes=(0, 0)))
    lap = np.where(prob.lap == 0.0, 1.0, prob.lap)
    psi_hat = np.where(prob.lap == 0.0, 0.0, 4.0 * math.pi * prob.lb * q_hat / lap)
    return np.real(fourier.idft3(psi_hat))


def screening_convolution(prob, rho):
    """sum_j (DC_ij (*) (rho_j - rho_bath_j))(x) for each species i (eq. muESexpansion)."""
    rho_hat = fourier.dft3(rho)
    drho_hat = rho_hat.copy()
    drho_hat[:, 0, 0, 0] -= prob.npoints * prob.bath.rho
    out = []
    for i in range(prob.nspecies):
        acc = np.zeros(prob.shape, dtype=np.complex128)
        for j in range(prob.nspecies):
            acc += prob.dc_hat[i][j] * drho_hat[j]
        out.append(acc)
    return np.real(fourier.idft3(np.stack(out)))


def mu_sc(prob, rho):
    """beta mu_SC_i(x) = beta mu_ES_bath_i - sum_j DC_ij (*) drho_j (eq. muESexpansion)."""
    return prob.bath.mu_es[:, None, None, None] - screening_convolution(prob, rho)


def c1_hs(prob, rho):
    """-beta mu_HS_i(x): the hard-sphere one-body direct correlation."""
    n = weighted_densities(prob, rho)
    return -mu_hs(prob, phi_derivative_fields(n, prob.functional))


def c1_es(prob, rho):
    """-(beta mu_SC_i(x) + z_i psi(x)), and psi itself."""
    p = psi(prob, rho)
    return -(mu_sc(prob, rho) + prob.z[:, None, None, None] * p[None]), p


def excess_mu(prob, rho):
    """beta mu_ex_i(x) = beta (mu_HS + mu_SC + z e phi) (eq. excessChemicalPotential)."""
    n = weighted_densities(prob, rho)
    return (mu_hs(prob, phi_derivative_fields(n, prob.functional)) + mu_sc(prob, rho)
            + prob.z[:, None, None, None] * psi(prob, rho)[None])


def picard_map(prob, rho, V):
    """G(rho) of eq. rhoEquation; V is beta mu_ext (S, Nz, Ny, Nx), +inf for hard exclusion.

    A fixed-number species i (n_fixed[i] > 0; the paper is silent on it, reading: the
    canonical form of eq. rhoEquation) has the same Boltzmann factor normalised to its
    particle number instead of the bath: G_i = N_i e_i / (h^3 sum_x e_i),
    e_i = exp(-V_i - beta mu_ex_i(x)).
    """
    mu = excess_mu(prob, rho)
    expo = prob.bath.mu_ex[:, None, None, None] - V - mu
    with np.errstate(over="ignore"):
        g = prob.bath.rho[:, None, None, None] * np.exp(expo)
    g = np.where(np.isinf(V), 0.0, g)
    for i in np.flatnonzero(prob.canonical):
        with np.errstate(over="ignore"):
            e = np.where(np.isinf(V[i]), 0.0, np.exp(-V[i] - mu[i]))
        g[i] = prob.n_fixed[i] * e / (prob.dv * np.sum(e))
    return g


def _accessible(V):
    return ~np.isinf(V)


def _require_grand_canonical(prob):
    if prob.canonical.any():
        raise NotImplementedError("the grand potential here is for species in contact with the bath only")


def grand_potential(prob, rho, V):
    """Omega / kT of the module docstring; rho must vanish where V = +inf."""
    _require_grand_canonical(prob)
    acc = _accessible(V)
    rb = prob.bath.rho[:, None, None, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        ideal = np.where(rho > 0.0, rho * (np.log(rho / rb) - 1.0), 0.0)
        ext = np.where(acc, rho * (V - prob.bath.mu_ex[:, None, None, None]), 0.0)
    n = weighted_densities(prob, rho)
    f_hs = np.sum(phi_field(n, prob.functional))
    q = np.tensordot(prob.z, rho, axes=(0, 0))
    f_mf = 0.5 * np.sum(q * psi(prob, rho))
    drho = rho - rb
    f_sc = (np.sum(prob.bath.mu_es * np.sum(drho, axis=(1, 2, 3)))
            - 0.5 * np.sum(drho * screening_convolution(prob, rho)))
    return prob.dv * (np.sum(ideal) + np.sum(ext) + f_hs + f_mf + f_sc)


def grad_omega_rho(prob, rho, V):
    """dOmega/drho_i(x) / kT on accessible voxels (0 elsewhere)."""
    _require_grand_canonical(prob)
    acc = _accessible(V)
    rb = prob.bath.rho[:, None, None, None]
    mu = excess_mu(prob, rho)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.log(rho / rb) + V - prob.bath.mu_ex[:, None, None, None] + mu
    return np.where(acc, prob.dv * g, 0.0)


def grad_omega_v(prob, rho):
    """Explicit partial dOmega/dV_i(x) = h^3 rho_i(x)."""
    return prob.dv * rho


def grad_omega_bulk(shape, h, radius, z, bulk_molar, rho, V, temperature_K=298.15, eps_r=78.5, rel=1e-3,
                    functional="rslt"):
    """dOmega/drho_bath_k / kT (kT nm^3) at fixed rho and V, by its definition: central differences
    of Omega over the bath density with steps rel*c_k and rel*c_k/2, Richardson-extrapolated.  The
    bath (mu_ex_bath, mu_ES_bath, Gamma) and the bulk-fluid kernel are recomputed at every
    displaced bath; the step in mol/L converts to nm^-3 by the molar factor."""
    c = np.asarray(bulk_molar, dtype=np.float64)
    out = np.zeros(len(c))
    for k in range(len(c)):
        base = rel * c[k] if c[k] > 0 else 1e-9
        est = []
        for step in (base, 0.5 * base):
            cp, cm = c.copy(), c.copy()
            cp[k] += step
            cm[k] = max(c[k] - step, 0.0)
            op = grand_potential(Problem(shape, h, radius, z, cp, temperature_K, eps_r, functional=functional),
                                 rho, V)
            om = grand_potential(Problem(shape, h, radius, z, cm, temperature_K, eps_r, functional=functional),
                                 rho, V)
            est.append((op - om) / (cp[k] - cm[k]))
        out[k] = (4.0 * est[1] - est[0]) / 3.0 / molar_to_per_nm3(1.0)
    return out
