"""Pins of the oracle's convolutions, electrostatics and fixed-point map against what the
paper and the mathematics fix (Sec. "Verification", closed forms, quadrature, brute force)."""
import math

import numpy as np
import pytest

from oracle import fourier, functional as F
from oracle.fmt import phi
from quadrature import ball_transform_radial, fmt_transforms_by_quadrature
from paper_0910_1531_gb300 import workloads


def _prob(shape=(8, 8, 8), h=0.1, radius=(0.095, 0.181), z=(1.0, -1.0), molar=(0.1, 0.1)):
    return F.Problem(shape, h, radius, z, molar)


def _coords(prob):
    nz, ny, nx = prob.shape
    hx, hy, hz = prob.h
    z, y, x = np.meshgrid(np.arange(nz) * hz, np.arange(ny) * hy, np.arange(nx) * hx, indexing="ij")
    return x, y, z


def test_unit_density_gives_fundamental_measures():
    # Sec. "Verification": constant unit density recovers the geometric measures.
    prob = _prob(shape=(6, 8, 10), h=(0.11, 0.09, 0.1), radius=(0.095, 0.099, 0.181),
                 z=(1, 2, -1), molar=(0.1, 0.01, 0.12))
    rho = np.ones((3,) + prob.shape)
    n = F.weighted_densities(prob, rho)
    R = prob.radius
    expect = [3.0, R.sum(), (4 * math.pi * R ** 2).sum(), (4 * math.pi * R ** 3 / 3).sum()] + [0.0] * 6
    for a in range(10):
        assert np.allclose(n[a], expect[a], rtol=1e-13, atol=1e-13), a


def test_bath_n3_is_volume_fraction():
    prob = _prob(radius=(0.095, 0.099, 0.181), z=(1, 2, -1), molar=(0.1, 0.01, 0.12))
    rb = prob.bath.rho
    rho = np.broadcast_to(rb[:, None, None, None], (3,) + prob.shape).copy()
    n3 = F.weighted_densities(prob, rho)[3]
    assert np.allclose(n3, np.sum(rb * 4 * math.pi * prob.radius ** 3 / 3), rtol=1e-13)


@pytest.mark.parametrize("jvec", [(1, 2, 3), (0, 0, 3), (4, 0, 0), (3, 4, 1), (9, 7, 6)])
def test_single_fourier_mode_against_quadrature(jvec):
    # rho_i = c_i + a_i cos(q.x + p) with q a grid wave vector gives
    # n_alpha = sum_i [c_i w_i(0) + a_i Re(w_i(-q) e^{i(q.x + p)})], with the weight transforms taken
    # from quadrature of eq. omegaDef's integrals (independent of the closed forms).
    # (no Nyquist index here: a real grid field cannot carry sin at the Nyquist frequency;
    # that case has its own test below)
    prob = _prob(shape=(8, 10, 11), h=(0.1, 0.12, 0.08))
    nz, ny, nx = prob.shape
    hx, hy, hz = prob.h
    jx, jy, jz = jvec
    q = np.array([fourier.wavenumbers(nx, hx)[jx], fourier.wavenumbers(ny, hy)[jy],
                  fourier.wavenumbers(nz, hz)[jz]])
    x, y, z = _coords(prob)
    phase = q[0] * x + q[1] * y + q[2] * z + 0.3
    c = np.array([0.06, 0.05])
    a = np.array([0.02, -0.01])
    rho = c[:, None, None, None] + a[:, None, None, None] * np.cos(phase)[None]
    n = F.weighted_densities(prob, rho)
    expect = np.zeros((10,) + prob.shape)
    for i, R in enumerate(prob.radius):
        w0 = fmt_transforms_by_quadrature(np.zeros(3), R)
        wq = fmt_transforms_by_quadrature(q, R)
        scal = [0, 1, 2, 3]
        for s in scal:
            expect[s] += c[i] * w0[s].real + a[i] * np.real(wq[s] * np.exp(1j * phase))
        for comp in range(3):
            # w(-q) = -w(q) for the odd vector weights
            expect[4 + comp] += a[i] * np.real(-wq[4][comp] * np.exp(1j * phase))
            expect[7 + comp] += a[i] * np.real(-wq[5][comp] * np.exp(1j * phase))
    for s in range(10):
        assert np.allclose(n[s], expect[s], rtol=1e-9, atol=1e-11), s


def test_nyquist_mode_has_no_vector_component():
    # rho = c + a cos(pi x / h): n3 varies along x but its gradient vanishes at every grid point,
    # so n_V2x = n_V1x = 0 (the real part of the complex inverse transform).
    prob = _prob(shape=(4, 4, 8))
    x, _, _ = _coords(prob)
    rho = 0.06 + 0.02 * np.cos(math.pi * x / prob.h[0])[None].repeat(2, 0)
    n = F.weighted_densities(prob, rho)
    assert np.ptp(n[3]) > 1e-5
    assert np.max(np.abs(n[4:10])) < 1e-15


def test_bruteforce_real_space_correlation():
    # eq. nDef as a direct sum n(y) = sum_x rho(x) K(x - y) with the periodic kernel K = IDFT(w_hat).
    prob = _prob(shape=(5, 6, 7), h=(0.1, 0.1, 0.1))
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.01, 0.1, (2,) + prob.shape)
    n = F.weighted_densities(prob, rho)
    nz, ny, nx = prob.shape
    comps = []
    for i in range(2):
        w0, w1, w2, w3, wV1, wV2 = prob.w[i]
        comps.append([w0, w1, w2, w3] + list(wV1) + list(wV2))
    for a in (0, 3, 5, 9):
        expect = np.zeros(prob.shape)
        for i in range(2):
            K = np.real(fourier.dft3_bruteforce(np.broadcast_to(comps[i][a], prob.shape), +1)) / rho[0].size
            for yz in range(nz):
                for yy in range(ny):
                    for yx in range(nx):
                        shifted = K[(np.arange(nz)[:, None, None] - yz) % nz,
                                    (np.arange(ny)[None, :, None] - yy) % ny,
                                    (np.arange(nx)[None, None, :] - yx) % nx]
                        expect[yz, yy, yx] += np.sum(rho[i] * shifted)
        assert np.allclose(n[a], expect, rtol=1e-10, atol=1e-13), a


def test_nv2_is_gradient_of_n3():
    # n_V2 = grad n3 for the eq. nDef sign convention; checked with 6th-order FD on a smooth field.
    prob = _prob(shape=(24, 24, 24), h=0.05)
    rho = workloads.random_density(prob.shape, 2, prob.bath.rho, 0.3, seed=11)
    # low-pass the field so finite differences are accurate
    rh = fourier.dft3(rho)
    rh *= np.exp(-(prob.kmag * 0.25) ** 2)
    rho = np.real(fourier.idft3(rh))
    n = F.weighted_densities(prob, rho)
    n3 = n[3]
    for axis, comp, hd in ((2, 7, prob.h[0]), (1, 8, prob.h[1]), (0, 9, prob.h[2])):
        r = lambda s: np.roll(n3, -s, axis)
        fd = (45 * (r(1) - r(-1)) - 9 * (r(2) - r(-2)) + (r(3) - r(-3))) / (60 * hd)
        assert np.max(np.abs(fd - n[comp])) < 1e-5 * np.max(np.abs(n[comp])) + 1e-12


def test_back_convolution_is_gradient_of_hard_sphere_free_energy():
    # eq. muHS is the functional derivative of F_HS = int Phi(n); on the grid
    # dF/drho_i(x) = h^3 mu_HS_i(x) exactly, with F = h^3 sum_y Phi(n(y)).
    prob = _prob(shape=(8, 8, 8), h=0.1)
    rho = workloads.random_density(prob.shape, 2, [3.0, 2.0], 0.4, seed=12)
    mu = F.mu_hs(prob, F.phi_derivative_fields(F.weighted_densities(prob, rho)))
    fhs = lambda r: prob.dv * np.sum(F.phi_field(F.weighted_densities(prob, r)))
    for (i, zz, yy, xx) in [(0, 1, 2, 3), (1, 7, 0, 4), (0, 5, 5, 5), (1, 2, 6, 1)]:
        eps = 1e-4 * rho[i, zz, yy, xx]
        vals = []
        for t in (-2, -1, 1, 2):
            r = rho.copy()
            r[i, zz, yy, xx] += t * eps
            vals.append(fhs(r))
        fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * eps)
        assert fd == pytest.approx(prob.dv * mu[i, zz, yy, xx], rel=1e-8)


def test_uniform_fluid_chemical_potential_is_percus_yevick():
    prob = _prob(radius=(0.095, 0.099, 0.181), z=(1, 2, -1), molar=(1.0, 0.3, 1.6))
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], (3,) + prob.shape).copy()
    mu = F.mu_hs(prob, F.phi_derivative_fields(F.weighted_densities(prob, rho)))
    for i in range(3):
        assert np.allclose(mu[i], prob.bath.mu_hs[i], rtol=1e-12)


def test_poisson_fd_laplacian_in_real_space():
    # eq. potentialSolution: -Lap_h psi = 4 pi lambda_B (q - mean q), and mean psi = 0 (eq. potentialConstraint).
    prob = _prob(shape=(8, 10, 12), h=(0.1, 0.07, 0.12))
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.0, 0.2, (2,) + prob.shape)
    p = F.psi(prob, rho)
    lap = sum((np.roll(p, 1, a) - 2 * p + np.roll(p, -1, a)) / hd ** 2
              for a, hd in ((2, prob.h[0]), (1, prob.h[1]), (0, prob.h[2])))
    q = rho[0] - rho[1]
    assert np.allclose(-lap, 4 * math.pi * prob.lb * (q - q.mean()), atol=1e-10)
    assert abs(p.mean()) < 1e-13


def test_poisson_gaussian_charge_matches_continuum():
    # A neutralised Gaussian charge of width s: away from the images the potential approaches
    # lambda_B Q erf(r / (sqrt 2 s)) / r, up to the FD/periodic corrections (loose check).
    from scipy.special import erf
    n, hh, s = 48, 0.05, 0.15
    prob = F.Problem((n, n, n), hh, [0.1], [1.0], [0.0])
    x, y, z = _coords(prob)
    c = n * hh / 2
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    Q = 1.0
    rho = Q * np.exp(-r * r / (2 * s * s)) / ((2 * math.pi * s * s) ** 1.5)
    p = F.psi(prob, rho[None])
    mask = (r > 0.3) & (r < 0.6)
    cont = prob.lb * Q * erf(r / (math.sqrt(2) * s)) / np.where(r > 0, r, 1.0)
    diff = (p - cont)[mask]
    # the periodic images and the zero-mean gauge shift the potential by a near-constant
    assert np.std(diff) < 0.02 * np.mean(cont[mask])


@pytest.mark.parametrize("jvec", [(1, 0, 0), (2, 3, 1)])
def test_screening_single_mode_against_quadrature(jvec):
    # rho_j = rho_bath_j + a_j cos(q.x): sum_j DC_ij (*) drho_j = sum_j DC_ij_hat(q) a_j cos(q.x), with
    # DC_ij_hat(q) by radial quadrature of eq. CplusPsiFunc.
    from oracle.weights import delta_c_real
    prob = _prob(shape=(8, 8, 8), h=0.08, molar=(0.5, 0.5))
    nz, ny, nx = prob.shape
    jx, jy, jz = jvec
    q = np.array([fourier.wavenumbers(nx, prob.h[0])[jx], fourier.wavenumbers(ny, prob.h[1])[jy],
                  fourier.wavenumbers(nz, prob.h[2])[jz]])
    x, y, z = _coords(prob)
    cq = np.cos(q[0] * x + q[1] * y + q[2] * z)
    a = [0.01, -0.02]
    rho = prob.bath.rho[:, None, None, None] + np.array(a)[:, None, None, None] * cq[None]
    got = F.screening_convolution(prob, rho)
    lam = prob.bath.lam
    for i in range(2):
        expect = np.zeros(prob.shape)
        for j in range(2):
            Rij = prob.radius[i] + prob.radius[j]
            kern = lambda r: float(delta_c_real(r, prob.z[i], prob.z[j], lam[i], lam[j], Rij, prob.lb))
            expect += ball_transform_radial(float(np.linalg.norm(q)), Rij, kern) * a[j] * cq
        assert np.allclose(got[i], expect, rtol=1e-9, atol=1e-13)


def test_bath_is_fixed_point_of_G():
    # Uniform bath without external field: Delta rho = 0, psi = 0 and mu_HS = mu_HS_bath, so G(rho_b) = rho_b.
    prob = _prob(radius=(0.095, 0.099, 0.181), z=(1, 2, -1), molar=(0.1, 0.01, 0.12))
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], (3,) + prob.shape).copy()
    g = F.picard_map(prob, rho, np.zeros_like(rho))
    assert np.allclose(g, rho, rtol=1e-12)


def test_grand_potential_gradient():
    # dOmega/drho_i(x) = h^3 [ln(rho/rho_b) + V - mu_ex_b + mu_ex(x)] (discrete, exact),
    # and the gradient vanishes on the G fixed point's defining equation.
    prob = _prob(shape=(8, 8, 8), h=0.1, molar=(0.5, 0.5))
    rho = workloads.random_density(prob.shape, 2, prob.bath.rho, 0.3, seed=21)
    V = 0.5 * workloads.random_density(prob.shape, 2, [1.0, 1.0], 0.5, seed=22)
    grad = F.grad_omega_rho(prob, rho, V)
    for (i, zz, yy, xx) in [(0, 1, 2, 3), (1, 6, 0, 7), (0, 4, 4, 4)]:
        eps = 1e-4 * rho[i, zz, yy, xx]
        vals = []
        for t in (-2, -1, 1, 2):
            r = rho.copy()
            r[i, zz, yy, xx] += t * eps
            vals.append(F.grand_potential(prob, r, V))
        fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * eps)
        assert fd == pytest.approx(grad[i, zz, yy, xx], rel=1e-6, abs=1e-10)
    # at rho = G(rho) the log-form gradient vanishes: check the identity pointwise on any rho
    g = F.picard_map(prob, rho, V)
    assert np.allclose(grad / prob.dv, np.log(rho / g), atol=1e-12)
