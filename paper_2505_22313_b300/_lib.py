"""ctypes view of libdoe.so (include/doe.h).  Argument marshalling only.

The library is required: if libdoe.so is missing or fails to load, every call raises.
There is no CPU or PyTorch fallback for any step of the path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libdoe.so"
DEBUG_LIB_PATH = _PKG / "libdoe_debug.so"  # every kernel index bounds-checked (DOE_DEBUG build)

DOE_OK = 0
DOE_EINVAL = -1
DOE_EUNSUPPORTED = -2
DOE_ENOWS = -3
DOE_ECUDA = -4
DOE_ETIMEDOUT = -5
DOE_ESCRATCH = -6
DOE_NOALLOC_SCRATCH_BYTES = 32 << 20
DOE_BANDLIMIT = 0x1
DOE_BANDLIMIT_CIRCULAR = 0x2
DOE_FAULT_WAIT_TIMEOUT = 0x1
DOE_FAULT_BOUNDS = 0x2
DOE_UPSAMPLE_SHIFT = 4  # flags bits 4-5: log2 of the upsampling factor of the heights
DOE_UPSAMPLE_LANCZOS3 = 0x40  # Lanczos-3 instead of nearest upsampling
DOE_OP_PROPAGATE, DOE_OP_PSF, DOE_OP_GRAD = 1, 2, 3
DOE_GRAD_L2_TARGET, DOE_GRAD_VJP = 0, 1

# every entry point declared in include/doe.h
EXPORTS = (
    "doe_init", "doe_workspace_bytes", "doe_propagate", "doe_psf", "doe_psf_many",
    "doe_workspace_bytes_many", "doe_grad", "doe_render", "doe_render_workspace_bytes",
    "doe_wiener", "doe_wiener_workspace_bytes", "doe_adam_step", "doe_radial_heights",
    "doe_radial_workspace_bytes", "doe_radial_grad",
    "doe_band_limits", "doe_band_limits_xy", "doe_debug_band_mask", "doe_strerror", "doe_trace_enable", "doe_trace_read",
    "doe_pass_name", "doe_launch_count", "doe_psf_noalloc", "doe_fault_status", "doe_debug_build",
    "doe_check_wait_timeout",
)


class DoeError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load().doe_strerror(code).decode() if code != 0 else "ok"
        super().__init__(f"{what}: {msg} (code {code})")


class Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("dx", ctypes.c_double),
        ("z", ctypes.c_double),
        ("n_lambda", ctypes.c_int32),
        ("lambda_", ctypes.POINTER(ctypes.c_double)),
        ("n_index", ctypes.POINTER(ctypes.c_double)),
        ("flags", ctypes.c_uint32),
        ("theta_x", ctypes.c_double),
        ("theta_y", ctypes.c_double),
        ("src_d", ctypes.c_double),
    ]


_lib = None


def load(path: Path | None = None) -> ctypes.CDLL:
    """The library (libdoe.so), loaded once per process."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(Path(path) if path else LIB_PATH)
    return _lib


def open_library(p: Path) -> ctypes.CDLL:
    """A separate handle on a build of the library (libdoe.so or the bounds-checked
    libdoe_debug.so) with the C signatures set."""
    if not p.exists():
        raise RuntimeError(f"{p.name} not built ({p}); run `python -m paper_2505_22313_b300.build`")
    lib = ctypes.CDLL(str(p))
    V = ctypes.c_void_p
    I = ctypes.c_int
    S = ctypes.c_size_t
    G = ctypes.POINTER(Geom)
    F = ctypes.c_void_p  # device float* / complex* / double*
    sig = {
        "doe_init": ([], I),
        "doe_workspace_bytes": ([G, I], S),
        "doe_workspace_bytes_many": ([I, G, I], S),
        "doe_propagate": ([G, F, F, F, V, S, V], I),
        "doe_psf": ([G, F, F, F, V, S, V], I),
        "doe_psf_many": ([I, G, ctypes.POINTER(V), ctypes.POINTER(V), ctypes.POINTER(V), V, S, V], I),
        "doe_grad": ([G, F, F, F, I, F, F, I, V, S, V], I),
        "doe_render": ([I, I, I, F, I, I, F, F, V, S, V], I),
        "doe_render_workspace_bytes": ([I, I, I], S),
        "doe_wiener": ([I, I, I, F, I, I, F, ctypes.c_double, F, V, S, V], I),
        "doe_wiener_workspace_bytes": ([I, I, I], S),
        "doe_adam_step": ([F, F, F, F, ctypes.c_longlong, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, I, ctypes.c_double, ctypes.c_double, V], I),
        "doe_radial_heights": ([I, F, I, F, V], I),
        "doe_radial_workspace_bytes": ([I], S),
        "doe_radial_grad": ([I, I, F, F, V, S, V], I),
        "doe_band_limits": ([G, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)], I),
        "doe_band_limits_xy": ([G, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int64)], I),
        "doe_debug_band_mask": ([G, I, F, V, S, V], I),
        "doe_strerror": ([I], ctypes.c_char_p),
        "doe_trace_enable": ([I], I),
        "doe_trace_read": ([I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)], I),
        "doe_pass_name": ([I], ctypes.c_char_p),
        "doe_launch_count": ([], ctypes.c_longlong),
        "doe_psf_noalloc": ([G, F, F, F, V], I),
        "doe_fault_status": ([ctypes.POINTER(ctypes.c_uint32)], I),
        "doe_debug_build": ([], I),
        "doe_check_wait_timeout": ([ctypes.c_uint32, V], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def check(code: int, what: str) -> None:
    if code != DOE_OK:
        raise DoeError(code, what)
