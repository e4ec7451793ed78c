"""The allocation-free weighted-density entry point agrees with the plan-based one.

Some callers cannot allocate device memory (a framework that has reserved the GPU's
memory for its own pool, code that must not trigger an allocation's implicit device
synchronisation, users who need a fixed device footprint); for them
dft_weighted_densities_noalloc keeps its scratch in a fixed device array inside the
library.  This file checks, through the C ABI, that two calls in a row (and a third on
another grid) give the same weighted densities as dft_weighted_densities, that the
largest documented case (64^3, five species) does too, that they match the FP64 oracle,
and that a grid too large for the fixed scratch is refused with a clear message.  It runs
last so that a failure here cannot hide the other tests; it passes alone or after them.
"""
import ctypes

import numpy as np
import pytest

from paper_0910_1531_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5   # the FP32 weighted-density tolerance of tests/test_gpu_parity.py
RADIUS = [0.095, 0.181]
VALENCE = [1.0, -1.0]
MOLAR = [0.5, 0.5]
# five species (radii nm, valences, molar), electroneutral
RADIUS5 = [0.095, 0.099, 0.181, 0.14, 0.12]
VALENCE5 = [1.0, 2.0, -1.0, -0.5, 0.0]
MOLAR5 = [0.1, 0.01, 0.1, 0.04, 0.3]
# the weighted densities alpha as index lists into the ten components (a vector is one field)
FIELDS = [[0], [1], [2], [3], [4, 5, 6], [7, 8, 9]]


@pytest.fixture(scope="module")
def lib():
    from paper_0910_1531_gb300 import binding, build
    build.build()
    return binding.load_library()


def _params(shape, h, radius, valence=VALENCE, molar=MOLAR):
    from paper_0910_1531_gb300.binding import DftParams
    keep = [np.array(radius, dtype=np.float64), np.array(valence[:len(radius)], dtype=np.float64),
            np.array(molar[:len(radius)], dtype=np.float64)]
    pd = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nz, ny, nx = shape
    prm = DftParams(nx, ny, nz, h, h, h, len(radius), pd(keep[0]), pd(keep[1]), pd(keep[2]), 298.15, 78.5, 0)
    return prm, keep


def _noalloc(lib, prm, rho, out):
    err = ctypes.create_string_buffer(512)
    st = lib.dft_weighted_densities_noalloc(ctypes.byref(prm), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                            ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            err, ctypes.sizeof(err))
    return st, err.value.decode()


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def test_matches_plan_entry_point_on_consecutive_calls(lib):
    from paper_0910_1531_gb300 import binding
    for shape, h, seed in (((32, 32, 32), 0.1, 1), ((32, 32, 32), 0.1, 2), ((24, 48, 16), 0.07, 3)):
        rho_np = workloads.random_density(shape, 2, [0.3, 0.3], 0.4, seed)
        rho = torch.tensor(rho_np, dtype=torch.float32, device="cuda")
        plan = binding.Plan(shape, h, RADIUS, VALENCE, MOLAR, precision="fp32")
        expect = plan.weighted_densities(rho).cpu().numpy()
        plan.close()
        prm, keep = _params(shape, h, RADIUS)
        out = torch.full((10,) + shape, float("nan"), dtype=torch.float32, device="cuda")
        st, msg = _noalloc(lib, prm, rho, out)
        assert st == 0, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for a in range(10):
            assert _relerr(got[a], expect[a]) < TOL, (shape, seed, a)


def test_rejects_a_grid_beyond_the_fixed_scratch(lib):
    shape = (128, 128, 128)
    prm, keep = _params(shape, 0.05, RADIUS)
    rho = torch.zeros((2,) + shape, dtype=torch.float32, device="cuda")
    out = torch.zeros((10,) + shape, dtype=torch.float32, device="cuda")
    st, msg = _noalloc(lib, prm, rho, out)
    assert st == -1
    assert "bytes of scratch" in msg


def test_largest_documented_case_matches_plan_entry_point(lib):
    # 64^3 with five species: (2 S + 10) half spectra of 64 x 64 x 34 points, 22.3 MB of the 24 MiB
    from paper_0910_1531_gb300 import binding
    shape, h = (64, 64, 64), 0.1
    rho_np = workloads.random_density(shape, 5, [0.06, 0.006, 0.06, 0.024, 0.18], 0.4, 5)
    rho = torch.tensor(rho_np, dtype=torch.float32, device="cuda")
    plan = binding.Plan(shape, h, RADIUS5, VALENCE5, MOLAR5, precision="fp32")
    expect = plan.weighted_densities(rho).cpu().numpy()
    plan.close()
    prm, keep = _params(shape, h, RADIUS5, VALENCE5, MOLAR5)
    for _ in range(2):
        out = torch.full((10,) + shape, float("nan"), dtype=torch.float32, device="cuda")
        st, msg = _noalloc(lib, prm, rho, out)
        assert st == 0, msg
        got = out.cpu().numpy()
        for a in range(10):
            assert _relerr(got[a], expect[a]) < TOL, a


def test_matches_the_oracle(lib):
    # the FP64 oracle's weighted densities (eq. nDef by eq. conv), per field alpha
    from oracle import functional as F
    shape, h = (24, 32, 20), (0.08, 0.1, 0.09)
    prob = F.Problem(shape, h, RADIUS, VALENCE, MOLAR)
    rho_np = workloads.random_density(shape, 2, prob.bath.rho, 0.4, 11)
    expect = F.weighted_densities(prob, rho_np)
    rho = torch.tensor(rho_np, dtype=torch.float32, device="cuda")
    prm, keep = _params(shape, h[0], RADIUS)
    prm.hx, prm.hy, prm.hz = h
    out = torch.full((10,) + shape, float("nan"), dtype=torch.float32, device="cuda")
    st, msg = _noalloc(lib, prm, rho, out)
    assert st == 0, msg
    got = out.cpu().numpy()
    for idx in FIELDS:
        assert _relerr(got[idx], expect[idx]) < TOL, idx


def test_limit_is_the_scratch_size(lib):
    # 72^3 (half spectra of 72 x 72 x 38 points): (2 S + 10) spectra fit in 24 MiB for two
    # species (22.1 MB) and not for three (25.2 MB)
    shape = (72, 72, 72)
    rho = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    out = torch.zeros((10,) + shape, dtype=torch.float32, device="cuda")
    prm, keep = _params(shape, 0.05, RADIUS)
    st, msg = _noalloc(lib, prm, rho, out)
    assert st == 0, msg
    prm3, keep3 = _params(shape, 0.05, RADIUS5[:3], VALENCE5[:3], [0.1, 0.01, 0.12])
    st, msg = _noalloc(lib, prm3, rho, out)
    assert st == -1
    assert "bytes of scratch" in msg
