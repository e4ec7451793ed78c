"""Pins of the Picard/line-search solver (Sec. "Nonlinear solver") and of its fixed point
(Sec. "Verification": homogeneity over planes parallel to a wall)."""
import math

import numpy as np
import pytest

from oracle import functional as F, picard
from paper_0910_1531_gb300 import workloads


def test_quadratic_alpha_recovers_parabola_minimum():
    f = lambda a: 3.0 * (a - 0.37) ** 2 + 0.1
    assert picard.quadratic_alpha(f(0), f(0.5), f(1.0), 1.0) == pytest.approx(0.37, rel=1e-14)
    g = lambda a: 2.0 * (a - 0.11) ** 2 + 0.5
    assert picard.quadratic_alpha(g(0), g(0.2), g(0.4), 0.4) == pytest.approx(0.11, rel=1e-14)
    # vertex beyond alpha_max -> alpha_max; vertex below the floor -> floor
    h = lambda a: (a - 3.0) ** 2
    assert picard.quadratic_alpha(h(0), h(0.5), h(1.0), 1.0) == 1.0
    k = lambda a: (a + 1.0) ** 2
    assert picard.quadratic_alpha(k(0), k(0.5), k(1.0), 1.0) == pytest.approx(1e-3)
    # concave: the better non-zero sample
    c = lambda a: -(a - 0.2) ** 2
    assert picard.quadratic_alpha(c(0), c(0.5), c(1.0), 1.0) == 1.0


def test_alpha_bound_is_the_printed_n3_bound():
    assert picard.alpha_bound(0.3, 0.2) == 1.0
    assert picard.alpha_bound(0.3, 0.6) == 1.0
    assert picard.alpha_bound(0.5, 1.3) == pytest.approx(0.5)
    # a step with alpha_max keeps (1 - a) M0 + a M1 at the bound
    a = picard.alpha_bound(0.45, 0.95)
    assert (1 - a) * 0.45 + a * 0.95 == pytest.approx(0.9)


def test_fixed_mixing_step():
    w = workloads.centred_sphere(n=8, h=0.1, molar=0.1, sphere_radius=0.2)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    g = F.picard_map(prob, rho0, w.V)
    rho1, info = picard.picard_step(prob, rho0, w.V, mixing=0.1)
    assert info["alpha"] == 0.1
    assert np.allclose(rho1, 0.9 * rho0 + 0.1 * g, rtol=1e-15)


def _wall_problem(molar=1.0):
    # Hard uncharged wall at z = 0 (zero thickness): a centre is excluded within R_i of the wall plane.
    shape, h = (32, 4, 4), (0.1, 0.1, 0.025)
    radius, z = np.array([0.1, 0.2125]), np.array([1.0, -1.0])
    prob = F.Problem(shape, h, radius, z, [molar, molar])
    zc = np.arange(shape[0]) * h[2]
    L = shape[0] * h[2]
    dist = np.minimum(zc, L - zc)
    V = np.zeros((2,) + shape)
    for i in range(2):
        V[i][dist < radius[i]] = np.inf
    return prob, V


def test_planar_wall_solution_is_homogeneous_over_planes():
    prob, V = _wall_problem()
    rho = np.where(np.isinf(V), 0.0, prob.bath.rho[:, None, None, None])
    rho, it, r = picard.solve(prob, rho, V, tol=0.0, max_it=15)
    plane_spread = np.max(np.ptp(rho, axis=(2, 3)))
    assert plane_spread < 1e-12 * np.max(rho)
    assert r < 1e-2   # the iteration makes progress from the bulk start


def test_line_search_converges_to_fixed_point():
    w = workloads.centred_sphere(n=12, h=0.1, molar=0.5, sphere_radius=0.25)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho = w.initial_rho_nm3(prob.bath.rho)
    rho, it, r = picard.solve(prob, rho, w.V, tol=1e-10, max_it=200)
    assert r < 1e-10
    g = F.picard_map(prob, rho, w.V)
    acc = ~np.isinf(w.V)
    assert np.max(np.abs(rho - g)[acc] / prob.bath.rho[np.nonzero(acc)[0]]) < 1e-8
    # a sphere centred on a grid point of a cubic grid: the solution is symmetric under axis swaps
    assert np.allclose(rho, np.swapaxes(rho, 1, 3), rtol=1e-9, atol=1e-14)
    assert np.allclose(rho, np.swapaxes(rho, 2, 3), rtol=1e-9, atol=1e-14)
    # and the gradient of Omega vanishes there
    grad = F.grad_omega_rho(prob, rho, w.V)
    assert np.max(np.abs(grad)) < 1e-8 * prob.dv


# ---- fixed-number (canonical) species: G_i = N_i e_i / (h^3 sum e_i) ----

def _pore(n=16, h=0.2):
    w = workloads.pore_slab_4species(n=n, h=h, o_count=8)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar, n_fixed=w.n_fixed)
    return w, prob


def test_canonical_species_holds_its_particle_number():
    w, prob = _pore()
    rho = w.initial_rho_nm3(prob.bath.rho)
    assert np.sum(rho[3]) * prob.dv == pytest.approx(8.0, rel=1e-14)
    g = F.picard_map(prob, rho, w.V)
    assert np.sum(g[3]) * prob.dv == pytest.approx(8.0, rel=1e-13)
    assert np.all(g[3][np.isinf(w.V[3])] == 0.0)
    # bath species are untouched by the fixed-number form
    gc = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    assert np.array_equal(g[:3], F.picard_map(gc, rho, w.V)[:3])


def test_canonical_equals_grand_canonical_at_the_same_number():
    # a species kept in the bath but marked fixed-number with N = h^3 sum of its grand-canonical
    # G has, by the normalisation alone, exactly the grand-canonical G
    w = workloads.centred_sphere(n=12, h=0.1, molar=0.3, sphere_radius=0.3)
    gc = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho = workloads.random_density(w.shape, 2, gc.bath.rho, 0.3, seed=5)
    rho = np.where(np.isinf(w.V), 0.0, rho)
    g_gc = F.picard_map(gc, rho, w.V)
    n1 = np.sum(g_gc[1]) * gc.dv
    can = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar, n_fixed=[0.0, n1])
    g_can = F.picard_map(can, rho, w.V)
    assert np.array_equal(g_can[0], g_gc[0])
    assert np.max(np.abs(g_can[1] - g_gc[1])) <= 1e-13 * np.max(g_gc[1])


def test_canonical_iteration_conserves_number_and_converges():
    w, prob = _pore()
    rho = w.initial_rho_nm3(prob.bath.rho)
    rho, it, r = picard.solve(prob, rho, w.V, tol=1e-6, max_it=60)
    assert np.sum(rho[3]) * prob.dv == pytest.approx(8.0, rel=1e-12)
    assert r < 1e-6
    # the weight of the residual is the species' mean density
    assert prob.rho_ref[3] == pytest.approx(8.0 / (prob.npoints * prob.dv))


def test_hard_wall_contact_sum_rule_under_refinement():
    # Sec. "Hard sphere fluids", eq. sumRule: at a hard wall the contact density of a hard-sphere
    # fluid equals the bath pressure, beta P = rho(R).  On the grid the contact value converges to
    # it at first order in h_z (the deviation halves with h_z); two Richardson steps (first- then
    # second-order) remove the discretisation error.  eta = 0.1, R = 0.1 nm, a 1.6 nm periodic
    # slit at h_z = 0.0125, 0.00625, 0.003125 nm.
    devs = []
    for nz, hz in ((128, 0.0125), (256, 0.00625), (512, 0.003125)):
        w = workloads.hard_wall_hs(0.1, nz=nz, nxy=2, hz=hz)
        prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
        rho0 = w.initial_rho_nm3(prob.bath.rho)
        rho, it, r = picard.solve(prob, rho0, w.V, tol=1e-11, max_it=200)
        assert r < 1e-11
        assert np.max(np.ptp(rho, axis=(2, 3))) < 1e-12 * np.max(rho)
        devs.append(rho[0, int(round(0.1 / hz)), 0, 0] / prob.bath.beta_p - 1.0)
    e1, e2, e3 = devs
    assert 1.9 < e1 / e2 < 2.1 and 1.9 < e2 / e3 < 2.1
    r1a, r1b = 2 * e2 - e1, 2 * e3 - e2
    assert abs((4 * r1b - r1a) / 3) < 1e-4
    assert abs(e2) > 0.01   # the unextrapolated value is off by about 1 %: the pin is the limit
