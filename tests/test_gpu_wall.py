"""The paper's representative ionic calculation (Sec. "Results"): 1 M univalent salt (cation
R 0.1 nm, anion R 0.2125 nm) at a hard, uncharged wall in a periodic 2 x 2 x 6 nm cell on a
21 x 21 x 161 grid.  The axis lengths 21 = 3 * 7 and 161 = 7 * 23 run through the odd-radix
stages of the run-time transforms.

Checks: G(rho) and the weighted densities against the oracle at the full size; the converged
solution (FP64) is homogeneous over planes parallel to the wall to rounding, as the paper reports
for its own solver, mirror-symmetric about the mid-plane of the periodic slit, and a fixed point of
the oracle's map; FP32 converges to the FP64 solution within the converged-density tolerance.
"""
import numpy as np
import pytest

from oracle import functional as F
from oracle import picard as P
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def wall():
    w = workloads.hard_wall_ionic()
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    return w, prob


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def plan_for(w, precision):
    from paper_0910_1531_gb300 import binding
    return binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision)


def to_dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wall_map_and_weighted_densities_match_oracle(wall, precision):
    w, prob = wall
    # a density with structure along all three axes, zero on the excluded voxels
    rho = workloads.random_density(w.shape, 2, prob.bath.rho, 0.3, seed=11)
    rho = np.where(np.isinf(w.V), 0.0, rho)
    plan = plan_for(w, precision)
    g_gpu, r_gpu = plan.picard_map(to_dev(rho, plan), to_dev(w.V, plan))
    g_ref = F.picard_map(prob, rho, w.V)
    assert relerr(g_gpu.cpu().numpy(), g_ref) < TOL[precision]
    r_ref = np.sqrt(P.residual_sq(prob, rho, g_ref))
    assert abs(r_gpu - r_ref) <= 10 * TOL[precision] * r_ref
    n_gpu = plan.weighted_densities(to_dev(rho, plan)).cpu().numpy()
    n_ref = F.weighted_densities(prob, rho)
    for a in range(10):
        assert relerr(n_gpu[a], n_ref[a]) < TOL[precision], a
    plan.close()


@pytest.fixture(scope="module")
def wall_fp64_solution(wall):
    w, prob = wall
    plan = plan_for(w, "fp64")
    rho = to_dev(w.initial_rho_nm3(prob.bath.rho), plan)
    it, r, ok = plan.solve(rho, to_dev(w.V, plan), tol=1e-9, max_it=3000)
    plan.close()
    assert ok, (it, r)
    return rho.cpu().numpy(), it


def test_wall_solution_is_planar_symmetric_and_a_fixed_point(wall, wall_fp64_solution):
    w, prob = wall
    rho, _ = wall_fp64_solution
    top = np.max(rho)
    # homogeneous over x-y planes
    assert np.max(np.ptp(rho, axis=(2, 3))) < 1e-12 * top
    # mirror symmetry of the periodic slit: z_k <-> z_(N-k)
    mirrored = np.roll(rho[:, ::-1], 1, axis=1)
    assert np.max(np.abs(rho - mirrored)) < 1e-10 * top
    # layering at the wall: the contact densities differ from the bath
    assert np.all(np.isfinite(rho))
    # a fixed point of the oracle's map (residual of the oracle at the GPU solution)
    g_ref = F.picard_map(prob, rho, w.V)
    assert np.sqrt(P.residual_sq(prob, rho, g_ref)) < 1e-8


def test_wall_fp32_converges_to_fp64_solution(wall, wall_fp64_solution):
    w, prob = wall
    ref, _ = wall_fp64_solution
    plan = plan_for(w, "fp32")
    rho = to_dev(w.initial_rho_nm3(prob.bath.rho), plan)
    it, r, ok = plan.solve(rho, to_dev(w.V, plan), tol=1e-5, max_it=3000)
    plan.close()
    assert ok, (it, r)
    got = rho.cpu().numpy()
    acc = ~np.isinf(w.V)
    for s in range(2):
        assert relerr(got[s][acc[s]], ref[s][acc[s]]) < 1e-4


# ---- hard spheres at a hard wall (Sec. "Hard sphere fluids", eq. sumRule) ----------------------

def _solve_fp64(w, tol=1e-10):
    from paper_0910_1531_gb300 import binding
    plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp64")
    beta_p = plan.bulk()["beta_p"]
    rho = torch.tensor(w.initial_rho_nm3(plan.bulk()["rho"]), dtype=torch.float64, device="cuda")
    V = torch.tensor(w.V, dtype=torch.float64, device="cuda")
    it, r, ok = plan.solve(rho, V, tol=tol, max_it=3000)
    if not ok:
        _, _, r, ok = plan.solve_newton(rho, V, tol, max_newton=100, krylov_dim=40)
    plan.close()
    assert ok, r
    return rho.cpu().numpy(), beta_p


@pytest.mark.parametrize("eta", [0.1, 0.3])
def test_hard_sphere_wall_contact_sum_rule(eta):
    # the contact density converges to beta P at first order in h_z; two Richardson steps leave
    # the sum rule satisfied to 1e-4
    devs = []
    for nz, hz in ((128, 0.0125), (256, 0.00625), (512, 0.003125)):
        w = workloads.hard_wall_hs(eta, nz=nz, hz=hz)
        rho, beta_p = _solve_fp64(w)
        assert np.max(np.ptp(rho, axis=(2, 3))) < 1e-12 * np.max(rho)
        devs.append(rho[0, int(round(0.1 / hz)), 0, 0] / beta_p - 1.0)
    e1, e2, e3 = devs
    assert 1.9 < e1 / e2 < 2.1 and 1.9 < e2 / e3 < 2.1
    assert abs((4 * (2 * e3 - e2) - (2 * e2 - e1)) / 3) < 1e-4


def test_hard_sphere_wall_solution_matches_oracle():
    w = workloads.hard_wall_hs(0.2, nz=128, hz=0.0125)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    ref, it, r = P.solve(prob, w.initial_rho_nm3(prob.bath.rho), w.V, tol=1e-11, max_it=300)
    assert r < 1e-11
    got, _ = _solve_fp64(w, tol=1e-11)
    acc = ~np.isinf(w.V)
    assert relerr(got[acc], ref[acc]) < 1e-9
