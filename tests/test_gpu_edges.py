"""Degenerate inputs and the error statuses the device reports (no GPU fault involved: the kernels
record a flag, the call returns the status, and the next call on the same plan works).

* rho = 0 everywhere: every weighted density is 0 and G is the bath's response to an empty box;
* a species excluded from every voxel: its G is 0 everywhere, the others match the oracle;
* a bath at packing fraction 0.6: the pointwise terms take the FP64 branch (n3 >= 0.5) and the
  uniform bath stays a fixed point;
* n3 >= 1 somewhere: DFT_EN3BOUND; an infinite Boltzmann factor: DFT_ENONFINITE;
* TMA tile waits bounded at 0 polls (each gives up at once): DFT_ETIMEOUT.
"""
import numpy as np
import pytest

from oracle import functional as F
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp64": 1e-10}
SHAPE = (16, 12, 18)
H = (0.1, 0.09, 0.11)
SPECIES = ([0.095, 0.181], [1.0, -1.0], [1.0, 1.0])


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def _plan(precision, species=SPECIES, shape=SHAPE, h=H):
    from paper_0910_1531_gb300 import binding
    return binding.Plan(shape, h, *species, precision=precision)


def _dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_empty_box(precision):
    prob = F.Problem(SHAPE, H, *SPECIES)
    rho = np.zeros((2,) + SHAPE)
    V = np.zeros_like(rho)
    plan = _plan(precision)
    n = plan.weighted_densities(_dev(rho, plan)).cpu().numpy()
    assert np.all(n == 0.0)
    g, _ = plan.picard_map(_dev(rho, plan), _dev(V, plan))
    assert relerr(g.cpu().numpy(), F.picard_map(prob, rho, V)) < TOL[precision]
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_species_excluded_everywhere(precision):
    prob = F.Problem(SHAPE, H, *SPECIES)
    rho = workloads.random_density(SHAPE, 2, prob.bath.rho, 0.3, seed=31)
    V = np.zeros_like(rho)
    V[1] = np.inf
    rho[1] = 0.0
    plan = _plan(precision)
    g, _ = plan.picard_map(_dev(rho, plan), _dev(V, plan))
    g = g.cpu().numpy()
    assert np.all(g[1] == 0.0)
    assert relerr(g, F.picard_map(prob, rho, V)) < TOL[precision]
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dense_bath_is_a_fixed_point(precision):
    eta, R = 0.6, 0.1
    molar = eta / (4.0 / 3.0 * np.pi * R ** 3) / 0.602214076
    species = ([R], [0.0], [molar])
    prob = F.Problem((12, 12, 12), 0.05, *species)
    plan = _plan(precision, species, (12, 12, 12), 0.05)
    rho = np.broadcast_to(prob.bath.rho[:, None, None, None], (1, 12, 12, 12)).copy()
    g, r = plan.picard_map(_dev(rho, plan), _dev(np.zeros_like(rho), plan))
    # G = rho_b exp(beta mu_b - beta mu_HS(x)): the exponential turns the absolute FP32 error of
    # beta mu_HS (about 40 kT at eta = 0.6, terms up to 1/(1 - n3)^3 = 16) into a relative one, so
    # FP32 is held to the converged-density bound here (measured 4.9e-5)
    tol = 1e-4 if precision == "fp32" else TOL[precision]
    assert relerr(g.cpu().numpy(), rho) < tol
    assert r < tol
    plan.close()


def test_n3_bound_and_nonfinite_are_reported_and_the_plan_recovers():
    from paper_0910_1531_gb300.binding import DftError
    prob = F.Problem(SHAPE, H, *SPECIES)
    plan = _plan("fp32")
    good = np.broadcast_to(prob.bath.rho[:, None, None, None], (2,) + SHAPE).copy()
    V = np.zeros_like(good)
    dense = good.copy()
    dense[:, 4:12, 3:9, 5:13] *= 100.0          # n3 well above 1 in the block
    with pytest.raises(DftError) as e:
        plan.picard_map(_dev(dense, plan), _dev(V, plan))
    assert e.value.status == -5                  # DFT_EN3BOUND
    Vbad = V.copy()
    Vbad[0, 8, 6, 9] = -1e30                     # exp(+1e30): an infinite Boltzmann factor
    with pytest.raises(DftError) as e:
        plan.picard_map(_dev(good, plan), _dev(Vbad, plan))
    assert e.value.status == -6                  # DFT_ENONFINITE
    g, r = plan.picard_map(_dev(good, plan), _dev(V, plan))
    assert relerr(g.cpu().numpy(), good) < 1e-5 and r < 1e-5
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bounded_wait_gives_up_and_the_plan_recovers(precision):
    # A y length with a compile-time TMA pass (32): with a bound of 0 polls every tile wait gives
    # up at once, each CTA drains the copies it has in flight (full bound) and stops, and the
    # call reports DFT_ETIMEOUT; with the default bound back, the same plan's next G and step
    # match the oracle.
    from paper_0910_1531_gb300.binding import DftError
    shape, h = (12, 32, 18), (0.1, 0.09, 0.11)
    prob = F.Problem(shape, h, *SPECIES)
    rho = workloads.random_density(shape, 2, prob.bath.rho, 0.3, seed=37)
    V = np.zeros_like(rho)
    plan = _plan(precision, shape=shape, h=h)
    plan.set_wait_polls(0)
    with pytest.raises(DftError) as e:
        plan.picard_map(_dev(rho, plan), _dev(V, plan))
    assert e.value.status == -8                  # DFT_ETIMEOUT
    plan.set_wait_polls(None)
    g, _ = plan.picard_map(_dev(rho, plan), _dev(V, plan))
    assert relerr(g.cpu().numpy(), F.picard_map(prob, rho, V)) < TOL[precision]
    plan.close()
