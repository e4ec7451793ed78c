"""The other hard-sphere free-energy densities (the original Rosenfeld and the White Bear forms,
dft_params.functional) against the oracle: weighted-density-to-c1 back-convolution, G(rho), the
bath values the plan computes on the host, the uniform bath as a fixed point, and the grand
potential with its gradients."""
import numpy as np
import pytest

from oracle import functional as F
from oracle import picard as P
from oracle.bulk import hs_bath_fmt
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp64": 1e-10}
KINDS = ["rosenfeld", "white_bear"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def _plan(shape, h, radius, z, molar, precision, kind):
    from paper_0910_1531_gb300 import binding
    return binding.Plan(shape, h, radius, z, molar, precision=precision, functional=kind)


def _dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


CASES = [
    ((16, 24, 32), (0.1, 0.08, 0.12), ([0.095, 0.181], [1.0, -1.0], [0.5, 0.5])),
    ((32, 32, 32), 0.05, ([0.095, 0.099, 0.181], [1.0, 2.0, -1.0], [0.1, 0.01, 0.12])),   # compile-time 32
    ((12, 18, 24), 0.07, ([0.1, 0.2125], [1.0, -1.0], [1.0, 1.0])),
]


def _case(shape, h, species, seed):
    radius, z, molar = species
    rho_b = F.Problem(shape, h, radius, z, molar).bath.rho
    rho = workloads.random_density(shape, len(radius), rho_b, 0.4, seed)
    hh = (h, h, h) if np.isscalar(h) else h
    L = np.array([shape[2] * hh[0], shape[1] * hh[1], shape[0] * hh[2]])
    rng = np.random.default_rng(seed + 100)
    centres = [tuple(rng.uniform(0, 1, 3) * L) for _ in range(2)]
    V = workloads.sphere_exclusion(shape, hh, radius, centres, [0.25, 0.15])
    return np.where(np.isinf(V), 0.0, rho), V


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape,h,species", CASES)
def test_c1_and_map_match_oracle(shape, h, species, kind, precision):
    radius, z, molar = species
    prob = F.Problem(shape, h, radius, z, molar, functional=kind)
    rho, V = _case(shape, h, species, seed=21)
    plan = _plan(shape, h, radius, z, molar, precision, kind)
    c1 = plan.c1_hs(_dev(rho, plan)).cpu().numpy()
    assert relerr(c1, F.c1_hs(prob, rho)) < TOL[precision]
    g_gpu, r_gpu = plan.picard_map(_dev(rho, plan), _dev(V, plan))
    g_ref = F.picard_map(prob, rho, V)
    assert relerr(g_gpu.cpu().numpy(), g_ref) < TOL[precision]
    r_ref = np.sqrt(P.residual_sq(prob, rho, g_ref))
    assert abs(r_gpu - r_ref) <= 10 * TOL[precision] * r_ref
    plan.close()


@pytest.mark.parametrize("kind", KINDS)
def test_bath_and_uniform_fixed_point_fp64(kind):
    radius, z, molar = [0.1, 0.2125], [1.0, -1.0], [1.0, 1.0]
    shape = (16, 16, 16)
    plan = _plan(shape, 0.1, radius, z, molar, "fp64", kind)
    b = plan.bulk()
    prob = F.Problem(shape, 0.1, radius, z, molar, functional=kind)
    assert np.allclose(b["mu_hs"], prob.bath.mu_hs, rtol=1e-12)
    assert b["beta_p"] == pytest.approx(prob.bath.beta_p, rel=1e-12)
    if kind == "white_bear":
        mu, p = hs_bath_fmt(prob.bath.rho, radius, kind)
        assert np.allclose(b["mu_hs"], mu, rtol=1e-12)
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], (2,) + shape).copy()
    g, r = plan.picard_map(_dev(rho, plan), _dev(np.zeros_like(rho), plan))
    assert relerr(g.cpu().numpy(), rho) < 1e-12
    assert r < 1e-12
    plan.close()


@pytest.mark.parametrize("kind", KINDS)
def test_grand_potential_and_gradients_fp64(kind):
    w = workloads.smooth_field_nacl(n=16, h=0.1, molar=0.5, seed=2)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar, functional=kind)
    rho = workloads.random_density(w.shape, 2, prob.bath.rho, 0.3, seed=9)
    plan = _plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, "fp64", kind)
    om, d_rho, d_V, d_bulk = plan.grad(_dev(rho, plan), _dev(w.V, plan))
    assert om == pytest.approx(F.grand_potential(prob, rho, w.V), rel=1e-10)
    assert relerr(d_rho.cpu().numpy(), F.grad_omega_rho(prob, rho, w.V)) < 1e-10
    ref_bulk = F.grad_omega_bulk(w.shape, w.h, w.radius, w.z, w.bulk_molar, rho, w.V, functional=kind)
    assert np.allclose(d_bulk, ref_bulk, rtol=1e-6, atol=0)
    plan.close()
