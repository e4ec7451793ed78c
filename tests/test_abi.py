"""CPU checks of the C-ABI library: it loads, exports every entry point declared in
include/gb300dft.h, and rejects invalid plans before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0910_1531_gb300 import build, binding
    build.build()
    return binding.load_library()


def declared_functions():
    with open(os.path.join(ROOT, "include", "gb300dft.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dft_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dft_plan_create", "dft_plan_destroy", "dft_weighted_densities", "dft_c1_hs", "dft_c1_es",
                     "dft_picard_step", "dft_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_0910_1531_gb300 import binding
    assert set(declared_functions()) <= set(binding.SIGNATURES)


def _params(nx=16, ny=16, nz=16, radius=(0.095, 0.181), z=(1.0, -1.0), molar=(0.1, 0.1), precision=0, functional=0):
    from paper_0910_1531_gb300.binding import DftParams
    arrs = [np.array(radius, dtype=np.float64), np.array(z, dtype=np.float64), np.array(molar, dtype=np.float64)]
    pd = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    prm = DftParams(nx, ny, nz, 0.1, 0.1, 0.1, len(radius), pd(arrs[0]), pd(arrs[1]), pd(arrs[2]), 298.15, 78.5,
                    precision, None, functional)
    return prm, arrs


@pytest.mark.parametrize("kw,code", [
    (dict(nx=74), -1),                     # 74 = 2 * 37: prime factor above 31
    (dict(nx=1024), -1),                   # above 512
    (dict(nx=2), -1),                      # below 4
    (dict(radius=(0.0, 0.181)), -1),       # R <= 0
    (dict(molar=(0.1, -0.1)), -1),         # negative concentration
    (dict(molar=(0.1, 0.2)), -2),          # not electroneutral
    (dict(molar=(60.0, 60.0)), -1),        # bath packing fraction >= 0.9
    (dict(precision=7), -1),
    (dict(functional=3), -1),              # unknown hard-sphere form
])
def test_plan_create_rejects_invalid_parameters(lib, kw, code):
    prm, keep = _params(**kw)
    handle = ctypes.c_void_p()
    st = lib.dft_plan_create(ctypes.byref(prm), None, ctypes.byref(handle))
    assert st == code
    assert handle.value is None
    assert len(lib.dft_last_error(None)) > 0


def test_null_arguments(lib):
    assert lib.dft_plan_create(None, None, None) == -1
    assert lib.dft_plan_destroy(None) == 0
    assert lib.dft_weighted_densities(None, None, None) == -1


@pytest.mark.parametrize("nx,ny,nz", [(21, 21, 161), (35, 22, 23), (10, 58, 124), (512, 4, 6)])
def test_plan_create_accepts_prime_factors_up_to_31(lib, nx, ny, nz):
    # lengths with the odd primes 5..31 (direct odd-radix stages) and up to 512 pass validation;
    # without a GPU the call then fails at the device set-up, never with DFT_EINVAL
    prm, keep = _params(nx=nx, ny=ny, nz=nz)
    handle = ctypes.c_void_p()
    st = lib.dft_plan_create(ctypes.byref(prm), None, ctypes.byref(handle))
    if handle.value:
        lib.dft_plan_destroy(handle)
    assert st != -1, lib.dft_last_error(None)
