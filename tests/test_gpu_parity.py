"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, per field f: max|f_gpu - f_oracle| / max|f_oracle| (a vector weighted density is one
field)
  FP32 (DFT_FP32_STAB): 1e-5 for weighted densities (the stated bound), c1 and G;
                        1e-4 for converged densities.
  FP64 (DFT_FP64):      1e-10.
"""
import numpy as np
import pytest

from oracle import functional as F
from oracle import picard as P
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp64": 1e-10}
# the weighted densities alpha as index lists into the ten components: a vector weighted density
# is one field (its error is measured against the largest of its three components)
FIELDS = [[0], [1], [2], [3], [4, 5, 6], [7, 8, 9]]
SPECIES = {
    1: ([0.1], [0.0], [2.0]),
    2: ([0.095, 0.181], [1.0, -1.0], [0.5, 0.5]),
    3: ([0.095, 0.099, 0.181], [1.0, 2.0, -1.0], [0.1, 0.01, 0.12]),
    5: ([0.095, 0.099, 0.181, 0.14, 0.12], [1.0, 2.0, -1.0, -0.5, 0.0], [0.1, 0.01, 0.1, 0.04, 0.3]),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def make_case(shape, h, nspec, seed, obstacles=True, amplitude=0.3):
    radius, z, molar = SPECIES[nspec]
    prob = F.Problem(shape, h, radius, z, molar)
    rho = workloads.random_density(shape, nspec, prob.bath.rho, amplitude, seed)
    V = np.zeros_like(rho)
    if obstacles:
        L = np.array([shape[2] * prob.h[0], shape[1] * prob.h[1], shape[0] * prob.h[2]])
        rng = np.random.default_rng(seed + 100)
        centres = [tuple(rng.uniform(0, 1, 3) * L) for _ in range(2)]
        V = workloads.sphere_exclusion(shape, prob.h, prob.radius, centres, [0.25, 0.15])
        rho = np.where(np.isinf(V), 0.0, rho)
    return prob, rho, V


def plan_for(prob, precision):
    from paper_0910_1531_gb300 import binding
    return binding.Plan(prob.shape, prob.h, prob.radius, prob.z,
                        [r / 0.602214076 for r in prob.bath.rho], precision=precision)


def to_dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


CASES = [
    ((8, 8, 8), 0.1, 2),
    ((128, 16, 96), (0.05, 0.1, 0.06), 2),   # compile-time z 128, x 96; run-time y 16
    ((32, 256, 128), (0.08, 0.04, 0.1), 3),  # compile-time z 32, y 256, x 128
    ((96, 96, 16), 0.1, 2),                  # compile-time z 96 and y 96 (TMA), run-time x 16
    ((48, 64, 48), 0.1, 2),                  # compile-time z 48, y 64, x 48
    ((16, 24, 32), (0.1, 0.08, 0.12), 2),
    ((12, 18, 24), 0.07, 3),
    ((27, 16, 9), 0.09, 2),        # odd x axis (no Nyquist), radix-3 z
    ((48, 48, 48), 0.1, 3),
    ((4, 6, 64), 0.05, 5),         # thin grid, five species
    ((6, 4, 12), 0.1, 1),          # single uncharged species (Gamma = 0)
    ((35, 21, 10), (0.1, 0.09, 0.11), 2),   # odd radices 5 and 7 (z 5*7, y 3*7, x 5*2)
    ((23, 22, 14), 0.08, 3),       # radix 23 (z), 11 (y), 7 (x)
    ((6, 4, 512), 0.05, 2),        # the longest axis accepted, on each pass: x 512
    ((4, 512, 6), 0.05, 2),        # y 512
    ((512, 6, 4), 0.05, 2),        # z 512
    ((256, 8, 12), 0.05, 3),       # compile-time z 256: the persistent z passes of the 256^3 workloads
    ((256, 6, 8), (0.1, 0.1, 0.03), 5),   # z 256 with five species (the largest ES tile set)
    ((64, 32, 48), 0.08, 2),       # compile-time z 64, y 32 (TMA), x 48
    ((12, 8, 256), 0.05, 2),       # compile-time x 256
    # odd y axes under the persistent z passes (no Nyquist row: every tile's y derivatives are
    # formed or folded with its own k_y)
    ((64, 15, 32), (0.1, 0.09, 0.1), 2),   # compile-time z 64, y 15 = 3 * 5, x 32
    ((128, 9, 16), 0.07, 3),               # compile-time z 128, y 9 = 3 * 3, x 16
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,h,nspec", CASES)
def test_weighted_densities(shape, h, nspec, precision):
    prob, rho, V = make_case(shape, h, nspec, seed=1)
    plan = plan_for(prob, precision)
    n_gpu = plan.weighted_densities(to_dev(rho, plan)).cpu().numpy()
    n_ref = F.weighted_densities(prob, rho)
    # per weighted density alpha: n0, n1, n2, n3 and the vectors nV1, nV2 as one field each
    for f in FIELDS:
        assert relerr(n_gpu[f], n_ref[f]) < TOL[precision], (f, relerr(n_gpu[f], n_ref[f]))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,h,nspec", CASES)
def test_c1_hard_sphere(shape, h, nspec, precision):
    prob, rho, V = make_case(shape, h, nspec, seed=2)
    plan = plan_for(prob, precision)
    c_gpu = plan.c1_hs(to_dev(rho, plan)).cpu().numpy()
    c_ref = F.c1_hs(prob, rho)
    for s in range(nspec):
        assert relerr(c_gpu[s], c_ref[s]) < TOL[precision], (s, relerr(c_gpu[s], c_ref[s]))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,h,nspec", [c for c in CASES if c[2] <= 4])
def test_c1_electrostatic_and_psi(shape, h, nspec, precision):
    prob, rho, V = make_case(shape, h, nspec, seed=3)
    plan = plan_for(prob, precision)
    c_gpu, psi_gpu = plan.c1_es(to_dev(rho, plan), want_psi=True)
    c_ref, psi_ref = F.c1_es(prob, rho)
    for s in range(nspec):
        assert relerr(c_gpu[s].cpu().numpy(), c_ref[s]) < TOL[precision]
    if np.max(np.abs(psi_ref)) > 0:
        assert relerr(psi_gpu.cpu().numpy(), psi_ref) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,h,nspec", CASES)
def test_picard_map(shape, h, nspec, precision):
    prob, rho, V = make_case(shape, h, nspec, seed=4)
    plan = plan_for(prob, precision)
    g_gpu, r_gpu = plan.picard_map(to_dev(rho, plan), to_dev(V, plan))
    g_ref = F.picard_map(prob, rho, V)
    assert relerr(g_gpu.cpu().numpy(), g_ref) < TOL[precision]
    r_ref = np.sqrt(P.residual_sq(prob, rho, g_ref))
    assert abs(r_gpu - r_ref) <= TOL[precision] * max(r_ref, 1e-30) * 10
    assert np.all(g_gpu.cpu().numpy()[np.isinf(V)] == 0.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_picard_map_full_size_obstacles(precision):
    # The 128^3 three-species workload the benchmark times, in the same launch configuration.
    w = workloads.obstacles_3species(n=128, h=0.05, seed=1)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho = w.initial_rho_nm3(prob.bath.rho)
    plan = plan_for(prob, precision)
    g_gpu, r_gpu = plan.picard_map(to_dev(rho, plan), to_dev(w.V, plan))
    g_ref = F.picard_map(prob, rho, w.V)
    assert relerr(g_gpu.cpu().numpy(), g_ref) < TOL[precision]
    r_ref = np.sqrt(P.residual_sq(prob, rho, g_ref))
    assert abs(r_gpu - r_ref) <= 1e-4 * r_ref
    n_gpu = plan.weighted_densities(to_dev(rho, plan)).cpu().numpy()
    n_ref = F.weighted_densities(prob, rho)
    for a in range(10):
        assert relerr(n_gpu[a], n_ref[a]) < TOL[precision], a


def test_uniform_bath_is_fixed_point_fp32():
    prob = F.Problem((32, 32, 32), 0.1, *SPECIES[3])
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], (3, 32, 32, 32)).copy()
    plan = plan_for(prob, "fp32")
    g, r = plan.picard_map(to_dev(rho, plan), to_dev(np.zeros_like(rho), plan))
    assert relerr(g.cpu().numpy(), rho) < 1e-5
    assert r < 1e-5


def test_fixed_mixing_trajectory_fp64():
    w = workloads.centred_sphere(n=16, h=0.1, molar=0.1, sphere_radius=0.3)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    plan = plan_for(prob, "fp64")
    rho = to_dev(rho0, plan)
    V = to_dev(w.V, plan)
    ref = rho0.copy()
    for it in range(10):
        r_gpu, a_gpu = plan.picard_step(rho, V, 0.1)
        ref, info = P.picard_step(prob, ref, w.V, mixing=0.1)
        assert a_gpu == pytest.approx(info["alpha"], abs=1e-14)
        assert r_gpu == pytest.approx(info["resid"], rel=1e-9)
    assert relerr(rho.cpu().numpy(), ref) < 1e-10


def test_line_search_steps_fp64():
    w = workloads.centred_sphere(n=16, h=0.1, molar=1.0, sphere_radius=0.3)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    plan = plan_for(prob, "fp64")
    rho = to_dev(rho0, plan)
    V = to_dev(w.V, plan)
    ref = rho0.copy()
    plan.iter_begin(rho, V)
    alpha_prev = None
    for it in range(4):
        r_gpu, a_gpu = plan.iter_step(rho, V, -1.0)
        ref, info = P.picard_step(prob, ref, w.V, alpha_prev=alpha_prev)
        alpha_prev = info["alpha"]
        assert r_gpu == pytest.approx(info["resid"], rel=1e-9)
        assert a_gpu == pytest.approx(info["alpha"], rel=1e-8)
        assert relerr(rho.cpu().numpy(), ref) < 1e-10


def test_solve_converges_to_oracle_fp32():
    w = workloads.centred_sphere(n=16, h=0.1, molar=0.5, sphere_radius=0.3)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    ref, it_ref, r_ref = P.solve(prob, rho0.copy(), w.V, tol=1e-10, max_it=300)
    assert r_ref < 1e-10
    plan = plan_for(prob, "fp32")
    rho = to_dev(rho0, plan)
    it, r, ok = plan.solve(rho, to_dev(w.V, plan), tol=1e-6, max_it=300)
    assert ok, (it, r)
    acc = ~np.isinf(w.V)
    got = rho.cpu().numpy()
    for s in range(2):
        assert relerr(got[s][acc[s]], ref[s][acc[s]]) < 1e-4


def test_host_buffer_step_matches_device_step():
    w = workloads.centred_sphere(n=16, h=0.1, molar=0.5, sphere_radius=0.3)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    plan = plan_for(prob, "fp32")
    rho_d = to_dev(rho0, plan)
    r1, a1 = plan.picard_step(rho_d, to_dev(w.V, plan), -1.0)
    rho_h = torch.tensor(rho0, dtype=torch.float32).pin_memory()
    V_h = torch.tensor(w.V, dtype=torch.float32).pin_memory()
    r2, a2 = plan.picard_step_host(rho_h, V_h, -1.0)
    assert r1 == r2 and a1 == a2
    assert torch.equal(rho_h, rho_d.cpu())
    # a second call (staged inputs overwritten, the step replayed from the cached graph)
    r1, a1 = plan.picard_step(rho_d, to_dev(w.V, plan), -1.0)
    r2, a2 = plan.picard_step_host(rho_h, V_h, -1.0)
    assert r1 == r2 and a1 == a2
    assert torch.equal(rho_h, rho_d.cpu())


def test_profile_counts_launches():
    prob, rho, V = make_case((16, 16, 16), 0.1, 2, seed=5)
    plan = plan_for(prob, "fp32")
    plan.profile_enable(True)
    plan.picard_map(to_dev(rho, plan), to_dev(V, plan))
    n, ms, by = plan.profile_read("xphi")
    assert n == 1 and ms > 0
    nc = 16 * 16 * 9
    assert by == 2 * 9 * nc * 8     # nine weighted-density spectra in and out
    n, ms, by = plan.profile_read("yfft")
    assert n == 4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_keeps_results(precision):
    # the autotuner changes the partition of the rows among blocks (G bitwise unchanged) and may
    # pick other transform kernels (the same arithmetic in another order: G within rounding,
    # a tenth of the parity tolerance), the residual only by the grouping of its sums
    prob, rho, V = make_case((32, 32, 32), 0.1, 3, seed=11)
    plan = plan_for(prob, precision)
    rd, Vd = to_dev(rho, plan), to_dev(V, plan)
    g0, r0 = plan.picard_map(rd, Vd)
    g0 = g0.clone()
    lines = plan.autotune(rd, Vd, reps=2)
    assert set(lines) == {"xfwd", "xphi", "xupdate"}
    assert all(v in (1, 2, 3, 4, 5, 6, 7, 8, 10, 11, 16) for v in lines.values())
    g1, r1 = plan.picard_map(rd, Vd)
    assert relerr(g1.cpu().numpy(), g0.cpu().numpy()) < 0.1 * TOL[precision], plan.tuning()
    assert abs(r1 - r0) <= (1e-6 if precision == "fp32" else 1e-11) * abs(r0)
    # a second plan of the same shape takes the cached choice
    plan2 = plan_for(prob, precision)
    assert plan2.autotune(rd, Vd, reps=2) == lines
    plan.close()
    plan2.close()


@pytest.mark.parametrize("workload", ["obstacles256", "pore256"])
def test_full_size_256_axis_permutation_and_shift(workload):
    # The 256^3 configurations in the launch configuration the benchmark times, checked through
    # properties that hold at any size: the discrete operator of a cubic box with equal spacings
    # commutes with exchanging the x and z axes (the x pass and the z pass then compute each
    # other's share of the same G) and with a circular shift of the grid.
    from paper_0910_1531_gb300 import binding
    if workload == "obstacles256":
        w = workloads.obstacles_3species(n=256, h=0.025, seed=1)
        plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp32")
    else:
        w = workloads.pore_slab_4species(n=256, h=0.05)
        plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp32", n_fixed=w.n_fixed)
    S = w.nspecies
    base = w.initial_rho_nm3(plan.bulk()["rho"])
    ref_rho = np.where(base > 0, base, 0.0)
    pert = workloads.random_density((64, 64, 64), S, np.ones(S), 0.2, seed=17)
    rho = np.where(np.isinf(w.V), 0.0, ref_rho * np.tile(pert, (1, 4, 4, 4)))
    # G = pref exp(mu0 - V + c): FP32 rounding of c turns into a relative error of G of about
    # |c| ulps; in the pore the bound species reach |c| ~ 10 (Ca2+ enriched ~1e4 fold)
    tol = 1e-5 if workload == "obstacles256" else 1e-4
    g0, r0 = plan.picard_map(to_dev(rho, plan), to_dev(w.V, plan))
    g0 = g0.cpu().numpy()
    assert np.all(np.isfinite(g0)) and np.all(g0[np.isinf(w.V)] == 0.0)
    t = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 3))
    g1, r1 = plan.picard_map(to_dev(t(rho), plan), to_dev(t(w.V), plan))
    assert relerr(g1.cpu().numpy(), t(g0)) < tol
    assert r1 == pytest.approx(r0, rel=tol)
    sh = lambda a: np.ascontiguousarray(np.roll(a, (37, -91, 128), axis=(1, 2, 3)))
    g2, r2 = plan.picard_map(to_dev(sh(rho), plan), to_dev(sh(w.V), plan))
    assert relerr(g2.cpu().numpy(), sh(g0)) < tol
    assert r2 == pytest.approx(r0, rel=tol)
    plan.close()
