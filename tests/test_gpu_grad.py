"""Differentiated form: dft_grad and the autograd wrapper against the oracle, finite
differences and the envelope theorem (re-solved equilibria)."""
import numpy as np
import pytest

from oracle import functional as F
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def _plan(w, precision):
    from paper_0910_1531_gb300 import binding
    return binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision)


def _dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


TOL = {"fp32": dict(omega=1e-5, field=1e-5, bulk=2e-3), "fp64": dict(omega=1e-10, field=1e-10, bulk=1e-6)}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("obstacle", [False, True])
def test_grad_matches_oracle(precision, obstacle):
    w = workloads.smooth_field_nacl(n=16, h=0.1, molar=0.5, seed=2)
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    V = w.V.copy()
    if obstacle:
        c = 16 * 0.1 / 2
        V = np.where(np.isinf(workloads.sphere_exclusion(w.shape, w.h, w.radius, [(c, c, c)], [0.3])), np.inf, V)
    rho = workloads.random_density(w.shape, 2, prob.bath.rho, 0.3, seed=9)
    rho = np.where(np.isinf(V), 0.0, rho)
    plan = _plan(w, precision)
    om, d_rho, d_V, d_bulk = plan.grad(_dev(rho, plan), _dev(V, plan))
    om_ref = F.grand_potential(prob, rho, V)
    assert om == pytest.approx(om_ref, rel=TOL[precision]["omega"])
    assert relerr(d_rho.cpu().numpy(), F.grad_omega_rho(prob, rho, V)) < TOL[precision]["field"]
    assert relerr(d_V.cpu().numpy(), F.grad_omega_v(prob, rho)) < TOL[precision]["field"]
    ref_bulk = F.grad_omega_bulk(w.shape, w.h, w.radius, w.z, w.bulk_molar, rho, V)
    assert np.allclose(d_bulk, ref_bulk, rtol=TOL[precision]["bulk"], atol=0)


def test_autograd_matches_finite_differences_fp64():
    from paper_0910_1531_gb300.autograd import grand_potential
    w = workloads.smooth_field_nacl(n=8, h=0.1, molar=0.5, seed=2)
    plan = _plan(w, "fp64")
    prob = F.Problem(w.shape, w.h, w.radius, w.z, w.bulk_molar)
    rho0 = workloads.random_density(w.shape, 2, prob.bath.rho, 0.3, seed=4)
    rho = _dev(rho0, plan).requires_grad_(True)
    V = _dev(w.V, plan).requires_grad_(True)
    bath = torch.tensor(plan.bulk()["rho"], dtype=torch.float64, requires_grad=True)
    om = grand_potential(plan, rho, V, bath)
    om.backward()
    rng = np.random.default_rng(3)
    for _ in range(6):
        i, zz, yy, xx = (int(rng.integers(0, s)) for s in (2, 8, 8, 8))
        for t, step in ((rho, 1e-6 * float(rho0[i, zz, yy, xx])), (V, 1e-4)):
            with torch.no_grad():
                vals = []
                for sgn in (+1, -1):
                    p = t.detach().clone()
                    p[i, zz, yy, xx] += sgn * step
                    args = (p, V.detach()) if t is rho else (rho.detach(), p)
                    vals.append(float(grand_potential(plan, *args)))
            fd = (vals[0] - vals[1]) / (2 * step)
            assert fd == pytest.approx(float(t.grad[i, zz, yy, xx]), rel=1e-6, abs=1e-12)
    ref_bulk = F.grad_omega_bulk(w.shape, w.h, w.radius, w.z, w.bulk_molar, rho0, w.V)
    assert np.allclose(bath.grad.numpy(), ref_bulk, rtol=1e-6)


def test_envelope_theorem_on_gpu_fp64():
    # At the equilibrium rho*, Omega*(V) and Omega*(rho_bath) re-solved on the GPU have derivatives
    # equal to the explicit partials dft_grad reports (dOmega/drho = 0 there).
    from paper_0910_1531_gb300 import binding
    w = workloads.smooth_field_nacl(n=32, h=0.1, molar=0.5, seed=2)
    plan = _plan(w, "fp64")
    rho_b = plan.bulk()["rho"]
    rho = _dev(w.initial_rho_nm3(rho_b), plan)
    V = _dev(w.V, plan)
    it, r, ok = plan.solve(rho, V, tol=1e-11, max_it=2000)
    assert ok, (it, r)
    _, d_rho, d_V, d_bulk = plan.grad(rho, V)
    assert float(d_rho.abs().max()) < 1e-9
    voxels = workloads.fd_voxels(w.shape, count=4, seed=3)
    for (zz, yy, xx) in voxels:
        for i in range(2):
            vals = []
            for sgn in (+1, -1):
                Vp = V.clone()
                Vp[i, zz, yy, xx] += sgn * 1e-4
                rp = rho.clone()
                plan.solve(rp, Vp, tol=1e-11, max_it=2000)
                vals.append(plan.grad(rp, Vp, want_rho=False, want_V=False, want_bulk=False)[0])
            fd = (vals[0] - vals[1]) / 2e-4
            assert fd == pytest.approx(float(d_V[i, zz, yy, xx]), rel=1e-5)
    # a plan needs an electroneutral bath: move both concentrations together and compare with the
    # derivative along that direction, sum_k dOmega/drho_bath_k
    vals = []
    dc = 1e-3 * w.bulk_molar[0]
    for sgn in (+1, -1):
        c = np.array(w.bulk_molar, dtype=float) + sgn * dc
        pk = binding.Plan(w.shape, w.h, w.radius, w.z, c, precision="fp64")
        rp = rho.clone()
        pk.solve(rp, V, tol=1e-11, max_it=2000)
        vals.append(pk.grad(rp, V, want_rho=False, want_V=False, want_bulk=False)[0])
        pk.close()
    total = (vals[0] - vals[1]) / (2 * dc) / 0.602214076
    assert total == pytest.approx(d_bulk[0] + d_bulk[1], rel=1e-4)
