"""Batched form: a ragged batch advanced by CUDA-graph replays reproduces, bit for bit, the same
state points iterated one plan at a time (same kernels, same launch configuration)."""
import numpy as np
import pytest

from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def _states():
    out = []
    for n, c, r in ((12, 0.05, 0.3), (32, 0.5, 0.5), (16, 1.0, 0.35), (48, 0.02, 0.9), (24, 0.2, 0.4)):
        w = workloads.centred_sphere(n=n, h=0.1, molar=c, sphere_radius=r, mixing=None)
        out.append(w)
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("alpha", [-1.0, 0.1])
def test_batch_matches_independent_plans(precision, alpha):
    from paper_0910_1531_gb300 import binding
    ws = _states()
    dt = torch.float64 if precision == "fp64" else torch.float32
    specs = [dict(shape=w.shape, h=w.h, radius=w.radius, valence=w.z, bulk_molar=w.bulk_molar) for w in ws]
    batch = binding.Batch(specs, precision=precision)
    rhos, Vs, refs = [], [], []
    for w in ws:
        plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision)
        r0 = torch.tensor(w.initial_rho_nm3(plan.bulk()["rho"]), dtype=dt, device="cuda")
        V = torch.tensor(w.V, dtype=dt, device="cuda")
        ref = r0.clone()
        plan.iter_begin(ref, V)
        for _ in range(6):
            plan.iter_step(ref, V, alpha, sync=False)
        r_ref, _ = plan.iter_step(ref, V, alpha)
        refs.append((ref, r_ref))
        plan.close()
        rhos.append(r0)
        Vs.append(V)
    batch.begin(rhos, Vs)
    batch.iterate(3, alpha, resid=False)
    resid = batch.iterate(4, alpha)          # graph reused across calls
    torch.cuda.synchronize()
    for (ref, r_ref), rho, r in zip(refs, rhos, resid):
        assert torch.equal(ref, rho)
        assert np.isfinite(r)
    batch.close()


def test_batch_state_with_steep_residual_converges():
    # 0.87 M NaCl around a 0.95 nm sphere in a 9.6 nm box: the residual grows much faster than
    # quadratically along the Picard segment; the adaptive sampled interval keeps the line search
    # converging (with the interval fixed at alpha_max it diverged).
    from paper_0910_1531_gb300 import binding
    w = workloads.batch_state_points(count=64, seed=4)[6]
    plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp32")
    rho = torch.tensor(w.initial_rho_nm3(plan.bulk()["rho"]), dtype=torch.float32, device="cuda")
    V = torch.tensor(w.V, dtype=torch.float32, device="cuda")
    plan.iter_begin(rho, V)
    res = [plan.iter_step(rho, V, -1.0)[0] for _ in range(40)]
    assert all(np.isfinite(res))
    assert res[-1] < 0.05 * res[0]
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("alpha", [-1.0, 0.1])
def test_iter_run_graph_matches_iter_step(precision, alpha):
    # dft_iter_run runs a captured iteration in an on-device loop (one graph launch per call,
    # the count kept on the device): the iterate must equal, bit for bit, the same number of
    # dft_iter_step calls (same kernels in the same order), over two calls of 2 and 3
    from paper_0910_1531_gb300 import binding
    w = workloads.centred_sphere(n=32, h=0.1, molar=0.5, sphere_radius=0.5, mixing=None)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision)
    r0 = torch.tensor(w.initial_rho_nm3(plan.bulk()["rho"]), dtype=dt, device="cuda")
    V = torch.tensor(w.V, dtype=dt, device="cuda")
    ref = r0.clone()
    plan.iter_begin(ref, V)
    for _ in range(5):
        plan.iter_step(ref, V, alpha, sync=False)
    r_ref = plan.iter_run(ref, V, 0)          # zero iterations: only the residual read-back
    got = r0.clone()
    plan.iter_begin(got, V)
    plan.iter_run(got, V, 2, alpha, sync=False)
    r_got = plan.iter_run(got, V, 3, alpha)   # graph reused across calls
    torch.cuda.synchronize()
    assert torch.equal(ref, got)
    assert r_ref == r_got and np.isfinite(r_got)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dependent_launch_is_bitwise_neutral(precision):
    # programmatic dependent launch only lets a pass become resident while the previous one
    # finishes; each pass waits for the kernels before it, so the iterates with and without it
    # agree bit for bit (eager steps, then the captured on-device loop; the 64^3 obstacle
    # geometry runs the compile-time persistent TMA passes over many waves)
    from paper_0910_1531_gb300 import binding
    w = workloads.obstacles_3species(n=64, h=0.1)
    dt = torch.float64 if precision == "fp64" else torch.float32
    outs = []
    for pdl in (False, True):
        plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision=precision)
        plan.set_dependent_launch(pdl)
        assert ("programmatic dependent" in plan.tuning()) == pdl, plan.tuning()
        r = torch.tensor(w.initial_rho_nm3(plan.bulk()["rho"]), dtype=dt, device="cuda")
        V = torch.tensor(w.V, dtype=dt, device="cuda")
        plan.iter_begin(r, V)
        for _ in range(2):
            plan.iter_step(r, V, -1.0, sync=False)
        resid = plan.iter_run(r, V, 3)
        torch.cuda.synchronize()
        outs.append((r, resid))
        plan.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and np.isfinite(outs[1][1])


def test_autotuned_batch_matches_autotuned_plans():
    # dft_batch_autotune gives each state the autotuner's choice for its grid (cached per grid,
    # species count and precision); the batch then advances every state exactly as an
    # independently autotuned plan does
    from paper_0910_1531_gb300 import binding
    ws = _states()[:3]
    dt = torch.float32
    specs = [dict(shape=w.shape, h=w.h, radius=w.radius, valence=w.z, bulk_molar=w.bulk_molar) for w in ws]
    fields = []
    for w in ws:
        probe = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp32")
        fields.append((torch.tensor(w.initial_rho_nm3(probe.bulk()["rho"]), dtype=dt, device="cuda"),
                       torch.tensor(w.V, dtype=dt, device="cuda")))
        probe.close()
    refs = []
    for w, (r0, V) in zip(ws, fields):
        plan = binding.Plan(w.shape, w.h, w.radius, w.z, w.bulk_molar, precision="fp32")
        plan.autotune(r0, V, reps=2)
        r = r0.clone()
        plan.iter_begin(r, V)
        for _ in range(3):
            plan.iter_step(r, V, -1.0, sync=False)
        torch.cuda.synchronize()
        refs.append(r)
        plan.close()
    batch = binding.Batch(specs, precision="fp32")
    rhos = [r0.clone() for r0, _ in fields]
    Vs = [V for _, V in fields]
    batch.autotune(rhos, Vs, reps=2)
    batch.begin(rhos, Vs)
    batch.iterate(3, -1.0, resid=False)
    torch.cuda.synchronize()
    for a, b in zip(rhos, refs):
        assert torch.equal(a, b)
    batch.close()
