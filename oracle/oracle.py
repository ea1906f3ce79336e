"""ctypes binding of the FP64 CPU oracle (``mhd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the benchmark use
this module to compute reference results.  The GPU library never imports it, and it imports nothing
from the GPU library.

Array conventions: real fields are float64 arrays of shape (N, N, N) indexed [z, y, x] with
x_i = 2*pi*i/N; vector fields are (3, N, N, N) with components (x, y, z).  Spectra are complex128
arrays of shape (N, N, N) indexed [kz, ky, kx] in FFT index order, forward-normalised by N^-3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_LIB = os.path.join(_HERE, "libmhd_oracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = ("rho", "mx", "my", "mz", "bx", "by", "bz")
DIAG_KEYS = ("ke", "me", "eint", "cross_hel", "mean_speed", "mean_bmag", "smax", "mean_rho",
             "mean_mx", "mean_my", "mean_mz", "mean_bx", "mean_by", "mean_bz", "divb_rms",
             "t", "dt", "step")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nu", ctypes.c_double), ("eta", ctypes.c_double),
                ("cs", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("cfl_adv", ctypes.c_double), ("cfl_visc", ctypes.c_double), ("integrator", ctypes.c_int),
                ("famp", ctypes.c_double), ("fa", ctypes.c_double), ("fb", ctypes.c_double), ("fc", ctypes.c_double),
                ("fkf", ctypes.c_int)]


def _declare(lib):
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.or_create.restype = P
    lib.or_create.argtypes = [ctypes.POINTER(_Params)]
    lib.or_destroy.argtypes = [P]
    lib.or_set_state.argtypes = [P, D, D, D]
    lib.or_get_state.argtypes = [P, D, D, D]
    lib.or_get_spectrum.argtypes = [P, ctypes.c_int, D]
    lib.or_set_spectrum.argtypes = [P, ctypes.c_int, D]
    lib.or_rhs.argtypes = [P, D, D, D]
    lib.or_rhs_spectrum.argtypes = [P, ctypes.c_int, D]
    lib.or_step.argtypes = [P, ctypes.c_int]
    lib.or_set_fixed_dt.argtypes = [P, ctypes.c_double]
    lib.or_get_history.argtypes = [P, ctypes.c_int, D, D, D, ctypes.POINTER(ctypes.c_int64)]
    lib.or_diagnostics.argtypes = [P, D]
    lib.or_fft1d.argtypes = [D, ctypes.c_int, ctypes.c_int]
    lib.or_fft3d.argtypes = [D, ctypes.c_int, ctypes.c_int]
    lib.or_forward.argtypes = [D, D, ctypes.c_int]
    lib.or_inverse.argtypes = [D, D, ctypes.c_int]
    lib.or_kmax.argtypes = [ctypes.c_int]
    lib.or_num_shells.argtypes = [ctypes.c_int]
    lib.or_tracer_field.argtypes = [P, ctypes.c_int, ctypes.c_int64, D, D]
    lib.or_tracers_set.argtypes = [P, ctypes.c_int64, D]
    lib.or_tracers_get.argtypes = [P, D, D]
    lib.or_spectra.argtypes = [P, ctypes.c_int, D, D, D]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def load_library(path: str):
    """Load another build of the same source (used by the tests that plant mistakes in a copy of
    the oracle to show that the pins catch them)."""
    return _declare(ctypes.CDLL(path))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _real(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _cplx(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def num_threads() -> int:
    return int(_load().or_num_threads())


def kmax(n: int) -> int:
    return int(_load().or_kmax(n))


def fft1d(a, sign: int) -> np.ndarray:
    """Unscaled radix-2 transform sum_j a_j exp(sign 2 pi i jk/n) of a 1D array."""
    out = np.array(a, dtype=np.complex128, copy=True)
    if _load().or_fft1d(_dp(out), out.size, int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return out


def fft3d(a, sign: int) -> np.ndarray:
    """Unscaled radix-2 3D transform of an (N, N, N) complex array."""
    out = np.array(a, dtype=np.complex128, copy=True)
    n = out.shape[0]
    if out.shape != (n, n, n) or _load().or_fft3d(_dp(out), n, int(sign)) != 0:
        raise ValueError("expected an (N, N, N) array with N a power of two")
    return out


def forward(f) -> np.ndarray:
    """fhat = N^-3 FFT(f) of a real (N, N, N) field."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[0]
    out = np.empty((n, n, n), dtype=np.complex128)
    if _load().or_forward(_dp(f), _dp(out), n) != 0:
        raise ValueError("bad size")
    return out


def inverse(fh) -> np.ndarray:
    """f = Re IFFT(fhat), unscaled."""
    fh = np.ascontiguousarray(fh, dtype=np.complex128)
    n = fh.shape[0]
    out = np.empty((n, n, n), dtype=np.float64)
    if _load().or_inverse(_dp(fh), _dp(out), n) != 0:
        raise ValueError("bad size")
    return out


class Oracle:
    """One solver instance of the oracle (see ``mhd_oracle.c`` for the method and readings)."""

    AB2, RK4, PC = 0, 1, 2

    def __init__(self, n: int, nu: float, eta: float, cs: float, dt: float = 0.0,
                 cfl_adv: float = 0.2, cfl_visc: float = 0.5, lib=None, integrator: int = 0,
                 forcing=None):
        """`forcing` = (amplitude, A, B, C, k_f) of the ABC body force, or None."""
        lib = lib if lib is not None else _load()
        self.n = int(n)
        famp, fa, fb, fc, fkf = forcing if forcing is not None else (0.0, 0.0, 0.0, 0.0, 1)
        self.params = _Params(self.n, float(nu), float(eta), float(cs), float(dt),
                              float(cfl_adv), float(cfl_visc), int(integrator),
                              float(famp), float(fa), float(fb), float(fc), int(fkf))
        self._h = lib.or_create(ctypes.byref(self.params))
        if not self._h:
            raise ValueError(f"oracle: cannot create instance (n={n} must be a power of two >= 4)")
        self._lib = lib

    def close(self):
        if self._h:
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.n, self.n, self.n)

    def set_state(self, rho, u, b):
        n = self.n
        rho = _real(rho, (n, n, n))
        u = _real(u, (3, n, n, n))
        b = _real(b, (3, n, n, n))
        self._lib.or_set_state(self._h, _dp(rho), _dp(u), _dp(b))

    def get_state(self):
        n = self.n
        rho = np.empty((n, n, n))
        m = np.empty((3, n, n, n))
        b = np.empty((3, n, n, n))
        self._lib.or_get_state(self._h, _dp(rho), _dp(m), _dp(b))
        return rho, m, b

    def spectrum(self, field: int) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        if self._lib.or_get_spectrum(self._h, int(field), _dp(out)) != 0:
            raise ValueError("bad field")
        return out

    def set_spectrum(self, field: int, spec) -> None:
        spec = _cplx(spec, self.shape)
        if self._lib.or_set_spectrum(self._h, int(field), _dp(spec)) != 0:
            raise ValueError("bad field")

    def rhs(self):
        n = self.n
        drho = np.empty((n, n, n))
        dm = np.empty((3, n, n, n))
        db = np.empty((3, n, n, n))
        self._lib.or_rhs(self._h, _dp(drho), _dp(dm), _dp(db))
        return drho, dm, db

    def rhs_spectrum(self, field: int) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        if self._lib.or_rhs_spectrum(self._h, int(field), _dp(out)) != 0:
            raise ValueError("bad field")
        return out

    def step(self, nsteps: int = 1) -> int:
        return int(self._lib.or_step(self._h, int(nsteps)))

    def set_fixed_dt(self, dt: float) -> None:
        """Take the following steps with step size `dt` (> 0), or with the CFL step (dt <= 0)."""
        if self._lib.or_set_fixed_dt(self._h, float(dt)) != 0:
            raise ValueError("bad step size")

    def history(self, field: int):
        out = np.empty(self.shape, dtype=np.complex128)
        dtp = ctypes.c_double()
        t = ctypes.c_double()
        st = ctypes.c_int64()
        self._lib.or_get_history(self._h, int(field), _dp(out), ctypes.byref(dtp), ctypes.byref(t),
                                 ctypes.byref(st))
        return out, dtp.value, t.value, st.value

    def diagnostics(self) -> dict:
        out = np.zeros(len(DIAG_KEYS))
        self._lib.or_diagnostics(self._h, _dp(out))
        d = dict(zip(DIAG_KEYS, out.tolist()))
        d["step"] = int(d["step"])
        d["etot"] = d["ke"] + d["me"] + d["eint"]
        return d

    def tracer_field(self, which: str, pos) -> np.ndarray:
        """CIC value of "B" or "u" at positions pos (count, 3)."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        out = np.zeros_like(pos)
        self._lib.or_tracer_field(self._h, 0 if which == "B" else 1, len(pos), _dp(pos), _dp(out))
        return out

    def tracers_set(self, pos) -> None:
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        self._ntr = len(pos)
        if self._lib.or_tracers_set(self._h, len(pos), _dp(pos)) != 0:
            raise RuntimeError("or_tracers_set failed")

    def tracers_get(self):
        """(positions, velocities), each (count, 3)."""
        n = getattr(self, "_ntr", 0)
        pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
        self._lib.or_tracers_get(self._h, _dp(pos), _dp(vel))
        return pos, vel

    def spectra(self) -> dict:
        """Shell spectra ek, em (index = shell), theta', S3, <d^2>, <d^3> of d = du_x/dx, the
        kinetic and magnetic helicities and max |div B| (see ``or_spectra``)."""
        ns = int(self._lib.or_num_shells(self.n))
        ek, em, st = np.zeros(ns), np.zeros(ns), np.zeros(7)
        rc = self._lib.or_spectra(self._h, ns, _dp(ek), _dp(em), _dp(st))
        if rc != 0:
            raise RuntimeError(f"or_spectra failed ({rc})")
        return {"ek": ek, "em": em, "theta": st[0], "s3": st[1], "d2": st[2], "d3": st[3],
                "kin_hel": st[4], "mag_hel": st[5], "divb_max": st[6]}
