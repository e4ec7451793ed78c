"""Every transform variant the autotuner can choose computes the same G as the oracle.

The x passes run either as the compile-time kernels (the Phi' passes one CTA per row block, or
persistent with bulk-copy or cp.async prefetch) or as the run-time ones under each candidate radix order
(default, reversed, all-8 and all-4 plans); the y pass as the persistent TMA kernel or
the run-time column kernel; the z passes as the persistent TMA kernels or the grouped
one-tile-per-CTA ones, the first half's z stage as one pass or three (z transforms around a
k-space products pass).  Each combination is pinned with dft_set_variants and checked against the
oracle's G (FP32 1e-5, FP64 1e-10), and one line-search step under a run-time x variant against
the oracle's step; finally dft_autotune's own choice is checked the same way.
"""
import numpy as np
import pytest

from oracle import functional as F
from oracle import picard as P
from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-5, "fp64": 1e-10}
SPECIES = ([0.095, 0.099, 0.181], [1.0, 2.0, -1.0], [0.1, 0.01, 0.12])


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0910_1531_gb300 import build
    build.build()


def relerr(a, b):
    b = np.asarray(b)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a) - b)) / (scale if scale > 0 else 1.0))


def _case(shape, h, seed):
    prob = F.Problem(shape, h, *SPECIES)
    rho = workloads.random_density(shape, 3, prob.bath.rho, 0.3, seed)
    L = np.array([shape[2] * prob.h[0], shape[1] * prob.h[1], shape[0] * prob.h[2]])
    V = workloads.sphere_exclusion(shape, prob.h, prob.radius, [tuple(0.4 * L)], [0.3])
    rho = np.where(np.isinf(V), 0.0, rho)
    return prob, rho, V


def _dev(x, plan):
    return torch.tensor(np.ascontiguousarray(x), dtype=plan.dtype, device="cuda")


def _x_variants(plan):
    """0 (compile-time, where the length has it) and 1.. (run-time radix orders) until refused."""
    from paper_0910_1531_gb300.binding import DftError
    out = []
    for x in range(0, 8):
        try:
            plan.set_variants(x, 0, 0)
        except DftError:
            if x == 0:
                continue
            break
        out.append(x)
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(32, 64, 128), (48, 32, 96)])
def test_every_variant_matches_oracle(precision, shape):
    from paper_0910_1531_gb300 import binding
    prob, rho, V = _case(shape, (0.05, 0.06, 0.07), seed=41)
    g_ref = F.picard_map(prob, rho, V)
    plan = binding.Plan(shape, prob.h, *SPECIES, precision=precision)
    xs = _x_variants(plan)
    assert len(xs) >= 3, xs            # compile-time and at least two radix orders
    for x in xs:
        for xp in ((0, 1) if x == 0 else (0,)):
            for y in (0, 1):
                for z in (0, 1, 2, 3):
                    plan.set_variants(x, y, z, x_persistent=xp)
                    g, _ = plan.picard_map(_dev(rho, plan), _dev(V, plan))
                    assert relerr(g.double().cpu().numpy(), g_ref) < TOL[precision], (x, xp, y, z, plan.tuning())
    plan.close()


@pytest.mark.parametrize("which", ["run-time", "persistent-bulk", "persistent-cp.async"])
def test_line_search_steps_under_variants_fp64(which):
    # three line-search iterations (paired samples, accepted point with its materialised
    # weighted densities) against the oracle's
    from paper_0910_1531_gb300 import binding
    shape = (32, 64, 128)
    prob, rho, V = _case(shape, (0.05, 0.06, 0.07), seed=43)
    ref = rho
    g = F.picard_map(prob, ref, V)
    a_prev = None
    for _ in range(3):
        ref, info = P.picard_step(prob, ref, V, g0=g, alpha_prev=a_prev)
        a_prev = info["alpha"]
        g = F.picard_map(prob, ref, V)
    plan = binding.Plan(shape, prob.h, *SPECIES, precision="fp64")
    if which == "run-time":
        plan.set_variants(_x_variants(plan)[-1], 1, 3)
    else:
        plan.set_variants(0, 0, 0, x_persistent=1 if which == "persistent-bulk" else 2)
    r, Vd = _dev(rho, plan), _dev(V, plan)
    plan.iter_begin(r, Vd)
    for _ in range(3):
        plan.iter_step(r, Vd, -1.0)
    assert relerr(r.cpu().numpy(), ref) < 1e-10, plan.tuning()
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotuned_choice_matches_oracle(precision):
    from paper_0910_1531_gb300 import binding
    shape = (32, 64, 128)
    prob, rho, V = _case(shape, (0.05, 0.06, 0.07), seed=47)
    plan = binding.Plan(shape, prob.h, *SPECIES, precision=precision)
    rd, Vd = _dev(rho, plan), _dev(V, plan)
    plan.autotune(rd, Vd, reps=2)
    desc = plan.tuning()
    assert desc.startswith("x: ") and "; y: " in desc and "; z: " in desc
    g, _ = plan.picard_map(rd, Vd)
    assert relerr(g.double().cpu().numpy(), F.picard_map(prob, rho, V)) < TOL[precision], desc
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(64, 32, 48), (128, 16, 32), (256, 8, 16)])
def test_split_first_half_equals_the_single_pass(precision, shape):
    # the three-pass first-half z stage (z transform, k-space products, z transform) runs the
    # same butterflies and the same products per point as the single pass; the compiler may
    # contract the products differently in the two kernels, so the weighted densities and G
    # agree to rounding (a few ulp of the largest value), and with the oracle
    from paper_0910_1531_gb300 import binding
    prob, rho, V = _case(shape, (0.05, 0.06, 0.07), seed=53)
    plan = binding.Plan(shape, prob.h, *SPECIES, precision=precision)
    rd, Vd = _dev(rho, plan), _dev(V, plan)
    out = []
    xv = _x_variants(plan)[0]       # the compile-time x kernels where the length has them
    for z in (0, 2):
        plan.set_variants(xv, 0, z)
        n = plan.weighted_densities(rd)
        g, _ = plan.picard_map(rd, Vd)
        out.append((n, g))
    close = {"fp32": 2e-6, "fp64": 1e-13}[precision]
    for a in range(2):
        assert relerr(out[1][a].double().cpu().numpy(), out[0][a].double().cpu().numpy()) < close, a
    assert relerr(out[1][1].double().cpu().numpy(), F.picard_map(prob, rho, V)) < TOL[precision]
    plan.close()
