"""Fixed-number (canonical) species on the GPU against the oracle: the pore/slab workload with
eight half-charged O confined to the pore (G_i = N_i e_i / (h^3 sum e_i))."""
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


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def setup(n=32, h=0.1, precision="fp32"):
    from paper_0910_1531_gb300 import binding
    w = workloads.pore_slab_4species(n=n, h=h)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar, n_fixed=w.n_fixed)
    plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision, n_fixed=w.n_fixed)
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")
    return w, prob, plan, dev


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n,h", [(32, 0.1), (48, 0.075)])
def test_canonical_picard_map_matches_oracle(precision, n, h):
    w, prob, plan, dev = setup(n, h, precision)
    rho = workloads.random_density(w.shape, 4, prob.rho_ref, 0.3, seed=7)
    rho = np.where(np.isinf(w.V), 0.0, rho)
    g_ref = F.picard_map(prob, rho, w.V)
    r_ref = np.sqrt(P.residual_sq(prob, rho, g_ref))
    g, r = plan.picard_map(dev(rho), dev(w.V))
    g = g.cpu().numpy()
    for i in range(4):
        assert relerr(g[i], g_ref[i]) < TOL[precision], i
    assert np.sum(g[3]) * prob.dv == pytest.approx(8.0, rel=10 * TOL[precision])
    assert r == pytest.approx(r_ref, rel=10 * TOL[precision])
    plan.close()


def test_canonical_line_search_trajectory_fp64():
    w, prob, plan, dev = setup(32, 0.1, "fp64")
    rho0 = w.initial_rho_nm3(prob.bath.rho)
    rho, V = dev(rho0), dev(w.V)
    ref = rho0.copy()
    plan.iter_begin(rho, V)
    alpha_prev = None
    for _ in range(4):
        r_gpu, a_gpu = plan.iter_step(rho, V, -1.0)
        ref, info = P.picard_step(prob, ref, w.V, alpha_prev=alpha_prev)
        alpha_prev = info["alpha"]
        assert r_gpu == pytest.approx(info["resid"], rel=1e-9)
        assert a_gpu == pytest.approx(info["alpha"], rel=1e-8)
    got = rho.cpu().numpy()
    assert relerr(got, ref) < 1e-10
    assert np.sum(got[3]) * prob.dv == pytest.approx(8.0, rel=1e-12)
    plan.close()


def test_canonical_iterations_fp32_conserve_number():
    w, prob, plan, dev = setup(32, 0.1, "fp32")
    rho = dev(w.initial_rho_nm3(prob.bath.rho))
    V = dev(w.V)
    plan.iter_begin(rho, V)
    res = [plan.iter_step(rho, V, -1.0)[0] for _ in range(20)]
    got = rho.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(res)) and res[-1] < res[0]
    assert np.sum(got[3]) * prob.dv == pytest.approx(8.0, rel=1e-5)
    assert np.all(got[3][np.isinf(w.V[3])] == 0.0)
    plan.close()


def test_grad_rejects_fixed_number_species():
    from paper_0910_1531_gb300 import binding
    w, prob, plan, dev = setup(16, 0.2, "fp32")
    rho = dev(w.initial_rho_nm3(prob.bath.rho))
    with pytest.raises(binding.DftError):
        plan.grad(rho, dev(w.V))
    plan.close()
