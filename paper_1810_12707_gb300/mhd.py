"""Python binding of the C ABI in ``include/mhd.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all numerical work runs in the
sm_103a kernels of ``libmhd_gb300.so``.  There is no fallback: if the library is missing or cannot
be loaded the first call raises.

Arrays: real fields are float64 (N, N, N) indexed [z, y, x]; vector fields (3, N, N, N).  Host
arrays are numpy arrays; device arrays are contiguous float64 CUDA torch tensors (passed as device
pointers with ``on_device = 1``).  PyTorch supplies the stream (its current stream at init) and,
by default, device memory through its caching allocator.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(_PKG, "libmhd_gb300.so")

MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_ESTATE, MHD_ENONFINITE, MHD_ETIMEOUT, MHD_EBUSY = range(8)
MHD_FP64 = 0
MHD_FP32_MIXED = 1
MHD_FP64_DF = 2
MHD_AB2, MHD_RK4, MHD_PC = 0, 1, 2
(MHD_OPT_CUDA_GRAPH, MHD_OPT_TILE_INV_Z, MHD_OPT_TILE_INV_Y, MHD_OPT_TILE_FWD_Y, MHD_OPT_TILE_FWD_Z,
 MHD_OPT_FLUX_PIPELINE, MHD_OPT_RADIX_INV_Z, MHD_OPT_RADIX_INV_Y, MHD_OPT_RADIX_FWD_Y,
 MHD_OPT_RADIX_FWD_Z, MHD_OPT_WAIT_POLLS, MHD_OPT_PERSISTENT, MHD_OPT_FUSED_UPDATE, MHD_OPT_TILE_FUSED) = range(14)
STATUS_NAMES = {0: "MHD_OK", 1: "MHD_EINVAL", 2: "MHD_ENOMEM", 3: "MHD_ECUDA", 4: "MHD_ESTATE",
                5: "MHD_ENONFINITE", 6: "MHD_ETIMEOUT", 7: "MHD_EBUSY"}

EXPORTS = ("mhd_footprint_bytes", "mhd_init", "mhd_destroy", "mhd_last_error", "mhd_set_state",
           "mhd_get_state", "mhd_rhs", "mhd_get_spectrum", "mhd_step", "mhd_synchronize",
           "mhd_diagnostics", "mhd_checkpoint_doubles", "mhd_checkpoint", "mhd_restore", "mhd_profile",
           "mhd_profile_read", "mhd_rhs_noalloc", "mhd_set_option", "mhd_pool_create", "mhd_pool_destroy",
           "mhd_pool_last_error", "mhd_pool_admit", "mhd_pool_step", "mhd_pool_progress",
           "mhd_pool_diagnostics", "mhd_pool_retire", "mhd_pool_info", "mhd_set_forcing", "mhd_num_shells",
           "mhd_spectra", "mhd_tracers_set", "mhd_tracers_get", "mhd_tracers_count", "mhd_autotune",
           "mhd_get_state_async")


class MhdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MhdParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("batch", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("dt", ctypes.c_double), ("cfl_adv", ctypes.c_double),
                ("cfl_visc", ctypes.c_double), ("stream", ctypes.c_void_p), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_user", ctypes.c_void_p)]


class MhdPhys(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("eta", ctypes.c_double), ("cs", ctypes.c_double)]


class MhdFlowStats(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("s3", ctypes.c_double), ("d2", ctypes.c_double),
                ("d3", ctypes.c_double), ("kin_hel", ctypes.c_double), ("mag_hel", ctypes.c_double),
                ("divb_max", ctypes.c_double)]


class MhdDiag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("ke", ctypes.c_double),
                ("me", ctypes.c_double), ("eint", ctypes.c_double), ("cross_hel", ctypes.c_double),
                ("mean_speed", ctypes.c_double), ("mean_bmag", ctypes.c_double), ("smax", ctypes.c_double),
                ("mean_rho", ctypes.c_double), ("mean_m", ctypes.c_double * 3), ("mean_b", ctypes.c_double * 3),
                ("divb_rms", ctypes.c_double), ("mach_s", ctypes.c_double), ("v_a", ctypes.c_double),
                ("mach_a", ctypes.c_double), ("step", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class MhdKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("total_ms", ctypes.c_double), ("launches", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIBRARY):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1810_12707_gb300.build_lib.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I32, D = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    lib.mhd_footprint_bytes.restype = ctypes.c_size_t
    lib.mhd_footprint_bytes.argtypes = [I32, I32, I32]
    lib.mhd_init.restype = I32
    lib.mhd_init.argtypes = [ctypes.POINTER(MhdParams), ctypes.POINTER(MhdPhys), ctypes.POINTER(P)]
    lib.mhd_destroy.restype = None
    lib.mhd_destroy.argtypes = [P]
    lib.mhd_last_error.restype = ctypes.c_char_p
    lib.mhd_last_error.argtypes = [P]
    for name in ("mhd_set_state", "mhd_get_state", "mhd_rhs"):
        fn = getattr(lib, name)
        fn.restype = I32
        fn.argtypes = [P, I32, P, P, P, I32]
    lib.mhd_get_state_async.restype = I32
    lib.mhd_get_state_async.argtypes = [P, I32, P, P, P]
    lib.mhd_get_spectrum.restype = I32
    lib.mhd_get_spectrum.argtypes = [P, I32, I32, P, I32]
    lib.mhd_step.restype = I32
    lib.mhd_step.argtypes = [P, I32]
    lib.mhd_synchronize.restype = I32
    lib.mhd_synchronize.argtypes = [P]
    lib.mhd_diagnostics.restype = I32
    lib.mhd_diagnostics.argtypes = [P, I32, ctypes.POINTER(MhdDiag)]
    lib.mhd_checkpoint_doubles.restype = ctypes.c_size_t
    lib.mhd_checkpoint_doubles.argtypes = [P]
    lib.mhd_checkpoint.restype = I32
    lib.mhd_checkpoint.argtypes = [P, I32, P, I32]
    lib.mhd_restore.restype = I32
    lib.mhd_restore.argtypes = [P, I32, P, I32]
    lib.mhd_profile.restype = I32
    lib.mhd_profile.argtypes = [P, I32]
    lib.mhd_profile_read.restype = I32
    lib.mhd_profile_read.argtypes = [P, ctypes.POINTER(MhdKernelTime), I32, ctypes.POINTER(I32)]
    lib.mhd_pool_create.restype = I32
    lib.mhd_pool_create.argtypes = [ctypes.POINTER(MhdParams), ctypes.POINTER(P)]
    lib.mhd_pool_destroy.restype = None
    lib.mhd_pool_destroy.argtypes = [P]
    lib.mhd_pool_last_error.restype = ctypes.c_char_p
    lib.mhd_pool_last_error.argtypes = [P]
    lib.mhd_pool_admit.restype = I32
    lib.mhd_pool_admit.argtypes = [P, ctypes.POINTER(MhdPhys), P, P, P, I32, ctypes.c_int64, ctypes.POINTER(I32)]
    lib.mhd_pool_step.restype = I32
    lib.mhd_pool_step.argtypes = [P, I32]
    lib.mhd_pool_progress.restype = I32
    lib.mhd_pool_progress.argtypes = [P, P, P, P]
    lib.mhd_pool_diagnostics.restype = I32
    lib.mhd_pool_diagnostics.argtypes = [P, I32, ctypes.POINTER(MhdDiag)]
    lib.mhd_pool_retire.restype = I32
    lib.mhd_pool_retire.argtypes = [P, I32, P, P, P, I32]
    lib.mhd_pool_info.restype = I32
    lib.mhd_pool_info.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.mhd_autotune.restype = I32
    lib.mhd_autotune.argtypes = [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]
    lib.mhd_tracers_set.restype = I32
    lib.mhd_tracers_set.argtypes = [P, I32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    lib.mhd_tracers_get.restype = I32
    lib.mhd_tracers_get.argtypes = [P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mhd_tracers_count.restype = ctypes.c_int64
    lib.mhd_tracers_count.argtypes = [P, I32]
    lib.mhd_num_shells.restype = I32
    lib.mhd_num_shells.argtypes = [I32]
    lib.mhd_spectra.restype = I32
    lib.mhd_spectra.argtypes = [P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), I32,
                                ctypes.POINTER(MhdFlowStats)]
    lib.mhd_set_forcing.restype = I32
    lib.mhd_set_forcing.argtypes = [P, I32, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, I32]
    lib.mhd_set_option.restype = I32
    lib.mhd_set_option.argtypes = [P, I32, ctypes.c_int64]
    lib.mhd_rhs_noalloc.restype = I32
    lib.mhd_rhs_noalloc.argtypes = [I32, ctypes.POINTER(MhdPhys), P, P, P, P, P, P, P]
    _lib = lib
    return lib


@dataclass
class Context:
    """An ``mhd_ctx*`` plus what must outlive it on the Python side."""
    handle: int
    n: int
    batch: int
    keepalive: tuple = ()

    def __del__(self):
        try:
            mhd_destroy(self)
        except Exception:
            pass


def _check(ctx, status: int):
    if status != MHD_OK:
        msg = load_library().mhd_last_error(ctx.handle if ctx is not None else None)
        raise MhdError(status, (msg or b"").decode())


def _torch():
    import torch
    return torch


def _is_device(a) -> bool:
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _in_ptr(a, shape):
    """(pointer, on_device, keepalive) of an input array."""
    if _is_device(a):
        torch = _torch()
        if a.dtype != torch.float64 or tuple(a.shape) != shape or not a.is_contiguous():
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")
        return a.data_ptr(), 1, a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.shape != shape:
        raise ValueError(f"expected shape {shape}, got {arr.shape}")
    return arr.ctypes.data, 0, arr


def _out(shape, device: bool, dtype=np.float64):
    if device:
        torch = _torch()
        t = torch.empty(shape, dtype=torch.float64 if dtype == np.float64 else torch.complex128, device="cuda")
        return t, t.data_ptr(), 1
    a = np.empty(shape, dtype=dtype)
    return a, a.ctypes.data, 0


def _torch_allocator():
    torch = _torch()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    @ALLOC_FN
    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:
            return None

    @FREE_FN
    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, free


def mhd_footprint_bytes(n: int, precision: int = MHD_FP64, batch: int = 1) -> int:
    return int(load_library().mhd_footprint_bytes(n, precision, batch))


def mhd_init(n: int, phys, dt: float = 0.0, cfl_adv: float = 0.2, cfl_visc: float = 0.5,
             precision: int = MHD_FP64, allocator: str = "torch", stream=None, integrator: int = MHD_AB2) -> Context:
    """Create a context; `phys` is a list of (nu, eta, cs), one per instance."""
    lib = load_library()
    phys = list(phys)
    arr = (MhdPhys * len(phys))(*[MhdPhys(float(a), float(b), float(c)) for a, b, c in phys])
    alloc = free = None
    keep = []
    if stream is None:
        try:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        except ImportError:
            stream = None
    if allocator == "torch":
        alloc, free = _torch_allocator()
        keep += [alloc, free]
    p = MhdParams(int(n), len(phys), int(precision), int(integrator), float(dt), float(cfl_adv), float(cfl_visc),
                  ctypes.c_void_p(stream) if stream else None,
                  alloc if alloc else ALLOC_FN(), free if free else FREE_FN(), None)
    h = ctypes.c_void_p()
    st = lib.mhd_init(ctypes.byref(p), arr, ctypes.byref(h))
    if st != MHD_OK:
        raise MhdError(st, "mhd_init failed")
    return Context(h.value, int(n), len(phys), tuple(keep))


def mhd_destroy(ctx: Context) -> None:
    if ctx.handle:
        load_library().mhd_destroy(ctx.handle)
        ctx.handle = 0


def mhd_set_state(ctx: Context, inst: int, rho, u, b) -> None:
    n = ctx.n
    pr, d0, k0 = _in_ptr(rho, (n, n, n))
    pu, d1, k1 = _in_ptr(u, (3, n, n, n))
    pb, d2, k2 = _in_ptr(b, (3, n, n, n))
    if not (d0 == d1 == d2):
        raise ValueError("inputs must all be host arrays or all device tensors")
    _check(ctx, load_library().mhd_set_state(ctx.handle, inst, pr, pu, pb, d0))


def _three_fields(ctx, fn, inst, device):
    n = ctx.n
    a, pa, dv = _out((n, n, n), device)
    b, pb, _ = _out((3, n, n, n), device)
    c, pc, _ = _out((3, n, n, n), device)
    _check(ctx, fn(ctx.handle, inst, pa, pb, pc, dv))
    return a, b, c


def mhd_get_state(ctx: Context, inst: int = 0, device: bool = False):
    """(rho, m, B) of one instance in real space."""
    return _three_fields(ctx, load_library().mhd_get_state, inst, device)


def mhd_get_state_async(ctx: Context, inst: int, rho: np.ndarray, m: np.ndarray, b: np.ndarray) -> None:
    """Queue the transfer of (rho, m, B) of one instance into host arrays of shapes (N,N,N),
    (3,N,N,N), (3,N,N,N), float64, C-contiguous (page-locked ones reach the link's rate); they are
    filled once mhd_synchronize returns and must stay alive until then."""
    n = ctx.n
    for a, shape in ((rho, (n, n, n)), (m, (3, n, n, n)), (b, (3, n, n, n))):
        if not (isinstance(a, np.ndarray) and a.shape == shape and a.dtype == np.float64 and a.flags.c_contiguous
                and a.flags.writeable):
            raise ValueError(f"need a writeable C-contiguous float64 host array of shape {shape}")
    _check(ctx, load_library().mhd_get_state_async(ctx.handle, int(inst), rho.ctypes.data, m.ctypes.data,
                                                   b.ctypes.data))


def mhd_rhs(ctx: Context, inst: int = 0, device: bool = False):
    """(d rho/dt, d m/dt, d B/dt) of one instance in real space, state unchanged."""
    return _three_fields(ctx, load_library().mhd_rhs, inst, device)


def mhd_get_spectrum(ctx: Context, inst: int, field: int, device: bool = False):
    """Spectrum of one state field, complex (N, N, N/2+1) indexed [kz, ky, kx]."""
    n = ctx.n
    out, p, dv = _out((n, n, n // 2 + 1), device, dtype=np.complex128)
    _check(ctx, load_library().mhd_get_spectrum(ctx.handle, inst, field, p, dv))
    return out


def mhd_step(ctx: Context, nsteps: int = 1) -> None:
    _check(ctx, load_library().mhd_step(ctx.handle, int(nsteps)))


def mhd_set_option(ctx: Context, option: int, value: int) -> None:
    _check(ctx, load_library().mhd_set_option(ctx.handle, int(option), int(value)))


def mhd_autotune(ctx: Context, reps: int = 5) -> dict:
    """Time every tile width (and, in the mixed mode, radix) of the four column FFT passes and
    keep the fastest; returns {"tiles": [4], "radix": [4], "ms": [4 mean ms per launch]} for
    (inverse z, inverse y, forward y, forward z)."""
    tiles = (ctypes.c_int32 * 4)()
    radix = (ctypes.c_int32 * 4)()
    ms = (ctypes.c_double * 4)()
    _check(ctx, load_library().mhd_autotune(ctx.handle, int(reps), tiles, radix, ms))
    return {"tiles": list(tiles), "radix": list(radix), "ms": list(ms)}


def mhd_tracers_set(ctx: Context, inst: int, pos) -> None:
    """Place tracers at pos (count, 3); their velocity starts as the interpolated grid velocity."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load_library().mhd_tracers_set(ctx.handle, int(inst), len(pos), pos.ctypes.data_as(dp)))


def mhd_tracers_get(ctx: Context, inst: int = 0):
    """(positions, velocities) of the tracers, each (count, 3)."""
    n = int(load_library().mhd_tracers_count(ctx.handle, int(inst)))
    if n < 0:
        raise MhdError(MHD_EINVAL, "bad context or instance")
    pos, vel = np.zeros((n, 3)), np.zeros((n, 3))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load_library().mhd_tracers_get(ctx.handle, int(inst), pos.ctypes.data_as(dp), vel.ctypes.data_as(dp)))
    return pos, vel


def mhd_num_shells(n: int) -> int:
    return int(load_library().mhd_num_shells(int(n)))


def mhd_spectra(ctx: Context, inst: int = 0) -> dict:
    """Shell spectra ek, em (index = shell round(|k|)), theta', S3, <d^2>, <d^3> of d = du_x/dx,
    the kinetic and magnetic helicities and max |div B|."""
    ns = mhd_num_shells(ctx.n)
    ek, em = np.zeros(ns), np.zeros(ns)
    st = MhdFlowStats()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load_library().mhd_spectra(ctx.handle, int(inst), ek.ctypes.data_as(dp), em.ctypes.data_as(dp), ns,
                                           ctypes.byref(st)))
    return {"ek": ek, "em": em, "theta": st.theta, "s3": st.s3, "d2": st.d2, "d3": st.d3,
            "kin_hel": st.kin_hel, "mag_hel": st.mag_hel, "divb_max": st.divb_max}


def mhd_set_forcing(ctx: Context, inst: int, amp: float, A: float = 1.0, B: float = 1.0, C: float = 1.0,
                    kf: int = 1) -> None:
    _check(ctx, load_library().mhd_set_forcing(ctx.handle, int(inst), float(amp), float(A), float(B), float(C), int(kf)))


def mhd_synchronize(ctx: Context) -> int:
    """Wait for queued work; returns MHD_OK or MHD_ENONFINITE (other statuses raise)."""
    st = load_library().mhd_synchronize(ctx.handle)
    if st not in (MHD_OK, MHD_ENONFINITE):
        _check(ctx, st)
    return st


def mhd_diagnostics(ctx: Context, inst: int = 0) -> dict:
    d = MhdDiag()
    _check(ctx, load_library().mhd_diagnostics(ctx.handle, inst, ctypes.byref(d)))
    out = {name: getattr(d, name) for name, _ in MhdDiag._fields_ if name not in ("mean_m", "mean_b", "reserved")}
    out["mean_m"] = list(d.mean_m)
    out["mean_b"] = list(d.mean_b)
    out["etot"] = d.ke + d.me + d.eint
    return out


def mhd_checkpoint_doubles(ctx: Context) -> int:
    return int(load_library().mhd_checkpoint_doubles(ctx.handle))


def mhd_checkpoint(ctx: Context, inst: int = 0) -> np.ndarray:
    buf = np.empty(mhd_checkpoint_doubles(ctx), dtype=np.float64)
    _check(ctx, load_library().mhd_checkpoint(ctx.handle, inst, buf.ctypes.data, 0))
    return buf


def mhd_restore(ctx: Context, inst: int, buf) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.float64)
    if buf.size != mhd_checkpoint_doubles(ctx):
        raise ValueError("checkpoint size does not match this context")
    _check(ctx, load_library().mhd_restore(ctx.handle, inst, buf.ctypes.data, 0))


def mhd_profile(ctx: Context, enable: bool) -> None:
    _check(ctx, load_library().mhd_profile(ctx.handle, 1 if enable else 0))


def mhd_profile_read(ctx: Context) -> dict:
    """{kernel name: (total device ms, launches)} accumulated while profiling was on."""
    arr = (MhdKernelTime * 16)()
    cnt = ctypes.c_int32()
    _check(ctx, load_library().mhd_profile_read(ctx.handle, arr, 16, ctypes.byref(cnt)))
    return {arr[i].name.decode(): (arr[i].total_ms, arr[i].launches) for i in range(cnt.value)}


def mhd_rhs_noalloc(n: int, phys, rho, u, b, stream=None):
    """RHS of one real-space state (CUDA float64 tensors) without any allocation inside the
    library (only the output tensors are allocated, here, by PyTorch).  n is 16 or 32.  Queued on
    `stream` (default: PyTorch's current stream); returns (drho, dm, dB) as CUDA tensors."""
    torch = _torch()
    shape3, shapev = (n, n, n), (3, n, n, n)
    args = []
    for a, shp in ((rho, shape3), (u, shapev), (b, shapev)):
        if not _is_device(a):
            raise ValueError("mhd_rhs_noalloc takes CUDA tensors")
        args.append(_in_ptr(a, shp)[0])
    outs = [torch.empty(shape3, dtype=torch.float64, device="cuda"),
            torch.empty(shapev, dtype=torch.float64, device="cuda"),
            torch.empty(shapev, dtype=torch.float64, device="cuda")]
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ph = MhdPhys(*[float(v) for v in phys])
    st = load_library().mhd_rhs_noalloc(int(n), ctypes.byref(ph), *args, *[o.data_ptr() for o in outs],
                                        ctypes.c_void_p(stream) if stream else None)
    if st != MHD_OK:
        raise MhdError(st, "mhd_rhs_noalloc failed")
    return tuple(outs)


# ---- serving pools ----

class Pool:
    """An ``mhd_pool*`` (see include/mhd.h): slots of one grid size stepped together."""

    def __init__(self, handle: int, n: int, slots: int, keepalive=()):
        self.handle, self.n, self.slots, self.keepalive = handle, n, slots, keepalive

    def __del__(self):
        try:
            mhd_pool_destroy(self)
        except Exception:
            pass


def _pcheck(pool, status: int):
    if status != MHD_OK:
        msg = load_library().mhd_pool_last_error(pool.handle)
        raise MhdError(status, (msg or b"").decode())


def mhd_pool_create(n: int, slots: int, dt: float = 0.0, cfl_adv: float = 0.2, cfl_visc: float = 0.5,
                    precision: int = MHD_FP32_MIXED, allocator: str = "torch", stream=None,
                    integrator: int = MHD_AB2) -> Pool:
    lib = load_library()
    keep = []
    alloc = free = None
    if stream is None:
        try:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        except ImportError:
            stream = None
    if allocator == "torch":
        alloc, free = _torch_allocator()
        keep += [alloc, free]
    p = MhdParams(int(n), int(slots), int(precision), int(integrator), float(dt), float(cfl_adv), float(cfl_visc),
                  ctypes.c_void_p(stream) if stream else None,
                  alloc if alloc else ALLOC_FN(), free if free else FREE_FN(), None)
    h = ctypes.c_void_p()
    st = lib.mhd_pool_create(ctypes.byref(p), ctypes.byref(h))
    if st != MHD_OK:
        raise MhdError(st, "mhd_pool_create failed")
    return Pool(h.value, int(n), int(slots), tuple(keep))


def mhd_pool_destroy(pool: Pool) -> None:
    if pool.handle:
        load_library().mhd_pool_destroy(pool.handle)
        pool.handle = 0


def mhd_pool_admit(pool: Pool, phys, rho, u, b, nsteps: int):
    """Admit a run; returns its slot handle, or None if every slot is busy."""
    n = pool.n
    pr, d0, k0 = _in_ptr(rho, (n, n, n))
    pu, d1, k1 = _in_ptr(u, (3, n, n, n))
    pb, d2, k2 = _in_ptr(b, (3, n, n, n))
    ph = MhdPhys(*[float(v) for v in phys])
    slot = ctypes.c_int32()
    st = load_library().mhd_pool_admit(pool.handle, ctypes.byref(ph), pr, pu, pb, d0, int(nsteps), ctypes.byref(slot))
    if st == MHD_EBUSY:
        return None
    _pcheck(pool, st)
    return slot.value


def mhd_pool_step(pool: Pool, k: int) -> None:
    _pcheck(pool, load_library().mhd_pool_step(pool.handle, int(k)))


def mhd_pool_progress(pool: Pool):
    """(steps, status, finished) arrays indexed by slot handle."""
    steps = np.zeros(pool.slots, dtype=np.int64)
    status = np.zeros(pool.slots, dtype=np.int32)
    fin = np.zeros(pool.slots, dtype=np.int32)
    _pcheck(pool, load_library().mhd_pool_progress(pool.handle, steps.ctypes.data, status.ctypes.data, fin.ctypes.data))
    return steps, status, fin


def mhd_pool_diagnostics(pool: Pool, slot: int) -> dict:
    d = MhdDiag()
    _pcheck(pool, load_library().mhd_pool_diagnostics(pool.handle, int(slot), ctypes.byref(d)))
    out = {name: getattr(d, name) for name, _ in MhdDiag._fields_ if name not in ("mean_m", "mean_b", "reserved")}
    out["etot"] = d.ke + d.me + d.eint
    return out


def mhd_pool_retire(pool: Pool, slot: int, copy_out: bool = True):
    """Free the slot; returns (rho, m, B) as numpy arrays (or None with copy_out=False)."""
    n = pool.n
    if copy_out:
        a = np.empty((n, n, n))
        m = np.empty((3, n, n, n))
        b = np.empty((3, n, n, n))
        _pcheck(pool, load_library().mhd_pool_retire(pool.handle, int(slot), a.ctypes.data, m.ctypes.data,
                                                      b.ctypes.data, 0))
        return a, m, b
    _pcheck(pool, load_library().mhd_pool_retire(pool.handle, int(slot), None, None, None, 0))
    return None


def mhd_pool_info(pool: Pool):
    live, mx = ctypes.c_int32(), ctypes.c_int32()
    _pcheck(pool, load_library().mhd_pool_info(pool.handle, ctypes.byref(live), ctypes.byref(mx)))
    return live.value, mx.value
