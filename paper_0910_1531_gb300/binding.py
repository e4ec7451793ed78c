"""Thin Python binding of libgb300dft.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/gb300dft.h with the same
name.  PyTorch supplies device memory and the CUDA stream; no arithmetic of the method
happens in Python.  If the library is missing or cannot be loaded, the first use raises
``RuntimeError`` -- there is no CPU fallback.
"""

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libgb300dft.so")
_lib = None
_lock = threading.Lock()

DFT_FP32_STAB = 0
DFT_FP64 = 1

STATUS = {0: "DFT_OK", -1: "DFT_EINVAL", -2: "DFT_ENONNEUTRAL", -3: "DFT_ENOMEM", -4: "DFT_ECUDA",
          -5: "DFT_EN3BOUND", -6: "DFT_ENONFINITE", -7: "DFT_ENOCONV", -8: "DFT_ETIMEOUT"}

WAIT_POLLS_DEFAULT = 1 << 24   # DFT_WAIT_POLLS_DEFAULT

KERNEL_NAMES = ("xfwd", "yfft", "zconv_fwd", "xphi", "zconv_bwd", "xupdate", "xinv", "finalize")


class DftError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class DftParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("nspecies", ctypes.c_int),
                ("radius_nm", ctypes.POINTER(ctypes.c_double)),
                ("valence", ctypes.POINTER(ctypes.c_double)),
                ("bulk_molar", ctypes.POINTER(ctypes.c_double)),
                ("temperature_K", ctypes.c_double), ("eps_r", ctypes.c_double),
                ("precision", ctypes.c_int),
                ("n_fixed", ctypes.POINTER(ctypes.c_double)),
                ("functional", ctypes.c_int)]

# dft_params.functional: the hard-sphere free-energy density (include/gb300dft.h, DFT_PHI_*)
FUNCTIONALS = {"rslt": 0, "rosenfeld": 1, "white_bear": 2}


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes): the entry points of include/gb300dft.h
SIGNATURES = {
    "dft_plan_create": (_I, [ctypes.POINTER(DftParams), _P, ctypes.POINTER(_P)]),
    "dft_plan_destroy": (_I, [_P]),
    "dft_last_error": (ctypes.c_char_p, [_P]),
    "dft_plan_bulk": (_I, [_P, _PD, _PD, _PD, _PD, _PD, _PD]),
    "dft_weighted_densities": (_I, [_P, _P, _P]),
    "dft_c1_hs": (_I, [_P, _P, _P]),
    "dft_c1_es": (_I, [_P, _P, _P, _P]),
    "dft_picard_map": (_I, [_P, _P, _P, _P, _PD]),
    "dft_picard_step": (_I, [_P, _P, _P, _D, _PD, _PD]),
    "dft_solve": (_I, [_P, _P, _P, _D, _D, _I, _PI, _PD]),
    "dft_iter_begin": (_I, [_P, _P, _P]),
    "dft_iter_step": (_I, [_P, _P, _P, _D, _PD, _PD]),
    "dft_iter_run": (_I, [_P, _P, _P, _I, _D, _PD]),
    "dft_solve_newton": (_I, [_P, _P, _P, _D, _I, _I, _PI, _PI, _PD]),
    "dft_autotune": (_I, [_P, _P, _P, _I, ctypes.POINTER(ctypes.c_int)]),
    "dft_picard_step_host": (_I, [_P, _P, _P, _D, _PD, _PD]),
    "dft_grad": (_I, [_P, _P, _P, _PD, _P, _P, _PD]),
    "dft_batch_create": (_I, [ctypes.POINTER(DftParams), _I, _P, ctypes.POINTER(_P)]),
    "dft_batch_destroy": (_I, [_P]),
    "dft_batch_last_error": (ctypes.c_char_p, [_P]),
    "dft_batch_begin": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "dft_batch_autotune": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I]),
    "dft_batch_iterate": (_I, [_P, _I, _D, _PD]),
    "dft_set_wait_polls": (_I, [_P, ctypes.c_longlong]),
    "dft_set_dependent_launch": (_I, [_P, _I]),
    "dft_plan_tuning": (ctypes.c_char_p, [_P]),
    "dft_set_variants": (_I, [_P, _I, _I, _I, _I]),
    "dft_profile_enable": (_I, [_P, _I]),
    "dft_profile_read": (_I, [_P, ctypes.c_char_p, _PI, _PD, _PD]),
    "dft_version": (ctypes.c_char_p, []),
    "dft_weighted_densities_noalloc": (_I, [ctypes.POINTER(DftParams), _P, _P, _P, ctypes.c_char_p, ctypes.c_size_t]),
}


def library_path():
    return _LIB_PATH


def load_library():
    """Load libgb300dft.so (raises RuntimeError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libgb300dft.so not built ({_LIB_PATH}); run paper_0910_1531_gb300.build.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """One state point: grid, species and bath; owns the library plan and its scratch."""

    def __init__(self, shape, h, radius, valence, bulk_molar, temperature_K=298.15, eps_r=78.5,
                 precision="fp32", stream=None, device=None, n_fixed=None, functional="rslt"):
        import torch
        self._torch = torch
        self.lib = load_library()
        nz, ny, nx = (int(v) for v in shape)
        if np.isscalar(h):
            h = (h, h, h)
        self.shape = (nz, ny, nx)
        self.h = tuple(float(v) for v in h)
        self.nspecies = len(radius)
        self.precision = DFT_FP64 if precision in ("fp64", DFT_FP64) else DFT_FP32_STAB
        self.dtype = torch.float64 if self.precision == DFT_FP64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._arrays = [np.ascontiguousarray(radius, dtype=np.float64),
                        np.ascontiguousarray(valence, dtype=np.float64),
                        np.ascontiguousarray(bulk_molar, dtype=np.float64)]
        if n_fixed is not None:
            self._arrays.append(np.ascontiguousarray(n_fixed, dtype=np.float64))
        pd = lambda a: a.ctypes.data_as(_PD)
        prm = DftParams(nx, ny, nz, self.h[0], self.h[1], self.h[2], self.nspecies,
                        pd(self._arrays[0]), pd(self._arrays[1]), pd(self._arrays[2]),
                        float(temperature_K), float(eps_r), self.precision,
                        pd(self._arrays[3]) if n_fixed is not None else None,
                        FUNCTIONALS[functional] if isinstance(functional, str) else int(functional))
        with torch.cuda.device(self.device):
            if stream is None:
                stream = torch.cuda.current_stream(self.device)
            self.stream = stream
            handle = ctypes.c_void_p()
            st = self.lib.dft_plan_create(ctypes.byref(prm), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(handle))
        if st != 0:
            raise DftError(st, self.lib.dft_last_error(None).decode())
        self.handle = handle

    # -- helpers -------------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise DftError(st, self.lib.dft_last_error(self.handle).decode())

    def _field(self, t, ncomp, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or not t.is_contiguous() or t.numel() != ncomp * self.npoints:
            raise ValueError(f"{name}: need contiguous {self.dtype} with {ncomp} x {self.shape} elements")
        return _ptr(t)

    @property
    def npoints(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def empty(self, ncomp):
        return self._torch.empty((ncomp,) + self.shape, dtype=self.dtype, device=self.device)

    # -- entry points --------------------------------------------------------------
    def bulk(self):
        S = self.nspecies
        rho, mh, me = (np.zeros(S) for _ in range(3))
        g, bp, lb = _D(), _D(), _D()
        self._check(self.lib.dft_plan_bulk(self.handle, rho.ctypes.data_as(_PD), mh.ctypes.data_as(_PD),
                                           me.ctypes.data_as(_PD), ctypes.byref(g), ctypes.byref(bp),
                                           ctypes.byref(lb)))
        return {"rho": rho, "mu_hs": mh, "mu_es": me, "gamma": g.value, "beta_p": bp.value, "lambda_b": lb.value}

    def weighted_densities(self, rho, out=None):
        out = self.empty(10) if out is None else out
        self._check(self.lib.dft_weighted_densities(self.handle, self._field(rho, self.nspecies, "rho"),
                                                    self._field(out, 10, "n_out")))
        return out

    def c1_hs(self, rho, out=None):
        out = self.empty(self.nspecies) if out is None else out
        self._check(self.lib.dft_c1_hs(self.handle, self._field(rho, self.nspecies, "rho"),
                                       self._field(out, self.nspecies, "c1_out")))
        return out

    def c1_es(self, rho, want_psi=False):
        out = self.empty(self.nspecies)
        psi = self.empty(1) if want_psi else None
        self._check(self.lib.dft_c1_es(self.handle, self._field(rho, self.nspecies, "rho"),
                                       self._field(out, self.nspecies, "c1_out"),
                                       self._field(psi, 1, "psi_out") if want_psi else None))
        return (out, psi[0]) if want_psi else out

    def picard_map(self, rho, V, out=None, resid=True):
        out = self.empty(self.nspecies) if out is None else out
        r = _D()
        self._check(self.lib.dft_picard_map(self.handle, self._field(rho, self.nspecies, "rho"),
                                            self._field(V, self.nspecies, "V"), self._field(out, self.nspecies, "g_out"),
                                            ctypes.byref(r) if resid else None))
        return (out, r.value) if resid else out

    def picard_step(self, rho, V, alpha=-1.0):
        r, a = _D(), _D()
        self._check(self.lib.dft_picard_step(self.handle, self._field(rho, self.nspecies, "rho"),
                                             self._field(V, self.nspecies, "V"), float(alpha),
                                             ctypes.byref(r), ctypes.byref(a)))
        return r.value, a.value

    def solve(self, rho, V, tol, max_it, alpha=-1.0, raise_on_noconv=False):
        it, r = _I(), _D()
        st = self.lib.dft_solve(self.handle, self._field(rho, self.nspecies, "rho"),
                                self._field(V, self.nspecies, "V"), float(alpha), float(tol), int(max_it),
                                ctypes.byref(it), ctypes.byref(r))
        if st == -7 and not raise_on_noconv:
            return it.value, r.value, False
        self._check(st)
        return it.value, r.value, True

    def solve_newton(self, rho, V, tol, max_newton=50, krylov_dim=30, raise_on_noconv=False):
        """Newton-Krylov solve in place; returns (newton steps, G evaluations, r, converged)."""
        it, ge, r = _I(), _I(), _D()
        st = self.lib.dft_solve_newton(self.handle, self._field(rho, self.nspecies, "rho"),
                                       self._field(V, self.nspecies, "V"), float(tol), int(max_newton),
                                       int(krylov_dim), ctypes.byref(it), ctypes.byref(ge), ctypes.byref(r))
        if st == -7 and not raise_on_noconv:
            return it.value, ge.value, r.value, False
        self._check(st)
        return it.value, ge.value, r.value, True

    def iter_begin(self, rho, V):
        self._check(self.lib.dft_iter_begin(self.handle, self._field(rho, self.nspecies, "rho"),
                                            self._field(V, self.nspecies, "V")))

    def iter_step(self, rho, V, alpha=-1.0, sync=True):
        r, a = _D(), _D()
        self._check(self.lib.dft_iter_step(self.handle, self._field(rho, self.nspecies, "rho"),
                                           self._field(V, self.nspecies, "V"), float(alpha),
                                           ctypes.byref(r) if sync else None, ctypes.byref(a) if sync else None))
        return (r.value, a.value) if sync else None

    def autotune(self, rho, V, reps=5):
        """Time the x-pass rows per block on these fields; returns {xfwd, xphi, xupdate} choices."""
        out = (ctypes.c_int * 3)()
        self._check(self.lib.dft_autotune(self.handle, self._field(rho, self.nspecies, "rho"),
                                          self._field(V, self.nspecies, "V"), int(reps), out))
        return {"xfwd": out[0], "xphi": out[1], "xupdate": out[2]}

    def iter_run(self, rho, V, iters, alpha=-1.0, sync=True):
        """`iters` iterations of iter_step as CUDA-graph replays; returns r after them (sync)."""
        r = _D()
        self._check(self.lib.dft_iter_run(self.handle, self._field(rho, self.nspecies, "rho"),
                                          self._field(V, self.nspecies, "V"), int(iters), float(alpha),
                                          ctypes.byref(r) if sync else None))
        return r.value if sync else None

    def grad(self, rho, V, want_rho=True, want_V=True, want_bulk=True):
        """(Omega, dOmega/drho, dOmega/dV, dOmega/drho_bath) through dft_grad; gradients None if not wanted."""
        om = _D()
        d_rho = self.empty(self.nspecies) if want_rho else None
        d_V = self.empty(self.nspecies) if want_V else None
        d_bulk = np.zeros(self.nspecies) if want_bulk else None
        self._check(self.lib.dft_grad(self.handle, self._field(rho, self.nspecies, "rho"),
                                      self._field(V, self.nspecies, "V"), ctypes.byref(om),
                                      self._field(d_rho, self.nspecies, "dOmega_drho") if want_rho else None,
                                      self._field(d_V, self.nspecies, "dOmega_dV") if want_V else None,
                                      d_bulk.ctypes.data_as(_PD) if want_bulk else None))
        return om.value, d_rho, d_V, d_bulk

    def picard_step_host(self, rho_host, V_host, alpha=-1.0):
        """rho_host, V_host: host tensors/arrays (pinned recommended) of the plan dtype; rho updated in place."""
        def hp(x):
            if isinstance(x, np.ndarray):
                assert x.flags["C_CONTIGUOUS"]
                return ctypes.c_void_p(x.ctypes.data)
            assert x.device.type == "cpu" and x.is_contiguous() and x.dtype == self.dtype
            return ctypes.c_void_p(x.data_ptr())
        r, a = _D(), _D()
        self._check(self.lib.dft_picard_step_host(self.handle, hp(rho_host), hp(V_host), float(alpha),
                                                  ctypes.byref(r), ctypes.byref(a)))
        return r.value, a.value

    def tuning(self):
        """The plan's transform variants, radix orders and rows per block, as one line of text."""
        return self.lib.dft_plan_tuning(self.handle).decode()

    def set_variants(self, x=0, y=0, z=0, x_persistent=0):
        """Pin the transform variants (see dft_set_variants)."""
        self._check(self.lib.dft_set_variants(self.handle, int(x), int(x_persistent), int(y), int(z)))

    def set_wait_polls(self, polls=None):
        """Bound of the y passes' TMA tile waits (None: the default); 0 makes them give up at once."""
        self._check(self.lib.dft_set_wait_polls(self.handle, WAIT_POLLS_DEFAULT if polls is None else int(polls)))

    def set_dependent_launch(self, enable=True):
        """Programmatic dependent launch of the passes (default on; see dft_set_dependent_launch)."""
        self._check(self.lib.dft_set_dependent_launch(self.handle, 1 if enable else 0))

    def profile_enable(self, enable=True):
        self._check(self.lib.dft_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self, name):
        """(launches, total ms, total algorithmic bytes) of one kernel kind since profile_enable."""
        n, ms, by = _I(), _D(), _D()
        self._check(self.lib.dft_profile_read(self.handle, name.encode(), ctypes.byref(n), ctypes.byref(ms),
                                              ctypes.byref(by)))
        return n.value, ms.value, by.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.dft_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Ragged batch of state points advanced together (one CUDA-graph launch per iteration).

    states: list of dicts with keys shape, h, radius, valence, bulk_molar (and optionally
    temperature_K, eps_r); all share `precision`.
    """

    def __init__(self, states, precision="fp32", stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.precision = DFT_FP64 if precision in ("fp64", DFT_FP64) else DFT_FP32_STAB
        self.dtype = torch.float64 if self.precision == DFT_FP64 else torch.float32
        self.states = []
        self._keep = []
        prms = (DftParams * len(states))()
        for i, st in enumerate(states):
            nz, ny, nx = st["shape"]
            h = st["h"]
            h = (h, h, h) if np.isscalar(h) else h
            arrs = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("radius", "valence", "bulk_molar")]
            if st.get("n_fixed") is not None:
                arrs.append(np.ascontiguousarray(st["n_fixed"], dtype=np.float64))
            self._keep.append(arrs)
            pd = lambda a: a.ctypes.data_as(_PD)
            prms[i] = DftParams(nx, ny, nz, h[0], h[1], h[2], len(arrs[0]), pd(arrs[0]), pd(arrs[1]), pd(arrs[2]),
                                float(st.get("temperature_K", 298.15)), float(st.get("eps_r", 78.5)), self.precision,
                                pd(arrs[3]) if len(arrs) > 3 else None)
            self.states.append((int(nz), int(ny), int(nx), len(arrs[0])))
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        handle = ctypes.c_void_p()
        st = self.lib.dft_batch_create(prms, len(states), ctypes.c_void_p(s.cuda_stream), ctypes.byref(handle))
        if st != 0:
            raise DftError(st, self.lib.dft_batch_last_error(None).decode())
        self.handle = handle
        self._ptrs = None

    def _check(self, st):
        if st != 0:
            raise DftError(st, self.lib.dft_batch_last_error(self.handle).decode())

    def _check_fields(self, rhos, Vs):
        for (nz, ny, nx, S), r, v in zip(self.states, rhos, Vs):
            for t in (r, v):
                if t.device.type != "cuda" or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != S * nz * ny * nx:
                    raise ValueError("batch field has the wrong shape, dtype or device")

    def autotune(self, rhos, Vs, reps=3):
        """Autotune every state's plan on its fields (dft_batch_autotune); call begin afterwards."""
        self._check_fields(rhos, Vs)
        n = len(self.states)
        rp = (_P * n)(*[r.data_ptr() for r in rhos])
        vp = (_P * n)(*[v.data_ptr() for v in Vs])
        self._check(self.lib.dft_batch_autotune(self.handle, rp, vp, int(reps)))

    def begin(self, rhos, Vs):
        self._check_fields(rhos, Vs)
        n = len(self.states)
        rp = (_P * n)(*[r.data_ptr() for r in rhos])
        vp = (_P * n)(*[v.data_ptr() for v in Vs])
        self._ptrs = (rp, vp, list(rhos), list(Vs))
        self._check(self.lib.dft_batch_begin(self.handle, rp, vp))

    def iterate(self, iters, alpha=-1.0, resid=True):
        out = np.zeros(len(self.states)) if resid else None
        self._check(self.lib.dft_batch_iterate(self.handle, int(iters), float(alpha),
                                               out.ctypes.data_as(_PD) if resid else None))
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.dft_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version():
    return load_library().dft_version().decode()
