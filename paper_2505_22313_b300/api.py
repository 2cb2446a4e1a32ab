"""PyTorch-facing API over libdoe.  Tensors supply device memory and the current CUDA
stream; every step of the computation runs in the library's CUDA kernels.

Notation (Wei et al. 2025, Sec. 3.1): h = DOE height map (metres), lambda = wavelength,
n = refractive index, z = propagation distance, dx = pitch, pad = zero-padding factor.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


@dataclass
class Geometry:
    """One DOE evaluation: N x N samples at pitch dx, padded to P = pad * N, at distance z,
    for the wavelengths `lambdas` with refractive indices `n_index`.  With upsample = f > 1 the
    heights (and the gradient) live on an (N / f) x (N / f) layout at pitch f dx, nearest-
    upsampled onto the simulation grid inside the first pass."""

    N: int
    dx: float
    z: float
    lambdas: np.ndarray
    n_index: np.ndarray
    pad: int = 2
    bandlimit: bool | str = True  # True: separable square band; "circular": the disc; False: none
    upsample: int = 1
    lanczos: bool = False  # Lanczos-3 instead of nearest upsampling of the layout
    theta_x: float = 0.0   # incident plane-wave tilt [rad]
    theta_y: float = 0.0
    src_d: float = 0.0     # spherical incident wave: source |d| before (> 0) / focus behind (< 0) [m]
    ny: int = 0            # rows of a rectangular DOE (0: square, N rows)

    @staticmethod
    def make(N, dx, z, lambdas, n_index=1.46, pad=2, bandlimit=True, upsample=1, lanczos=False,
             theta_x=0.0, theta_y=0.0, src_d=0.0, Ny=None) -> "Geometry":
        """N: the DOE's columns (x side); Ny: its rows (default N: a square DOE)."""
        lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lambdas, np.float64)))
        nid = np.ascontiguousarray(np.broadcast_to(np.asarray(n_index, np.float64), lam.shape).copy())
        if upsample not in (1, 2, 4, 8):
            raise ValueError("upsample must be 1, 2, 4 or 8")
        if isinstance(bandlimit, str) and bandlimit != "circular":
            raise ValueError("bandlimit must be True, False or 'circular'")
        bl = bandlimit if isinstance(bandlimit, str) else bool(bandlimit)
        return Geometry(int(N), float(dx), float(z), lam, nid, int(pad), bl, int(upsample), bool(lanczos),
                        float(theta_x), float(theta_y), float(src_d), int(Ny) if Ny is not None else 0)

    @property
    def Ny(self) -> int:
        """Rows of the DOE (y side)."""
        return self.ny or self.N

    @property
    def Py(self) -> int:
        """Rows of the padded grid."""
        return self.pad * self.Ny

    @property
    def NLy(self) -> int:
        """Rows of the height layout."""
        return self.Ny // self.upsample

    @property
    def NL(self) -> int:
        """Side of the height layout (N / upsample)."""
        return self.N // self.upsample

    @property
    def P(self) -> int:
        """Columns of the padded grid (its side on square grids)."""
        return self.pad * self.N

    @property
    def L(self) -> int:
        return int(self.lambdas.size)

    def c(self) -> L.Geom:
        g = L.Geom()
        g.nx = self.N
        g.ny = self.Ny
        g.pad = self.pad
        g.dx = self.dx
        g.z = self.z
        g.n_lambda = self.L
        g.lambda_ = self.lambdas.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        g.n_index = self.n_index.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        g.flags = ((L.DOE_BANDLIMIT if self.bandlimit else 0) | (L.DOE_BANDLIMIT_CIRCULAR if self.bandlimit == "circular" else 0)
                   | ((self.upsample.bit_length() - 1) << L.DOE_UPSAMPLE_SHIFT)
                   | (L.DOE_UPSAMPLE_LANCZOS3 if self.lanczos else 0))
        g.theta_x, g.theta_y, g.src_d = self.theta_x, self.theta_y, self.src_d
        return g


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t: torch.Tensor | None, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def workspace_bytes(geom: Geometry, op: int = L.DOE_OP_PSF) -> int:
    g = geom.c()
    return int(L.load().doe_workspace_bytes(ctypes.byref(g), op))


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device buffer usable as a libdoe workspace (the caching allocator aligns to 512 B)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def _ws_args(ws: torch.Tensor | None, need: int, device):
    if ws is None:
        ws = workspace(need, device)
    if ws.numel() < need:
        raise ValueError(f"workspace too small: {ws.numel()} < {need} bytes")
    return ws, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def init() -> None:
    L.check(L.load().doe_init(), "doe_init")


def psf(h: torch.Tensor, geom: Geometry, e_in: torch.Tensor | None = None, out: torch.Tensor | None = None,
        ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """PSFs I_lambda = |E_dest|^2 on the padded grid: float32 [L, Py, Px]."""
    hp = _dev_ptr(h, torch.float32, (geom.NLy, geom.NL), "h")
    ep = _dev_ptr(e_in, torch.complex64, (geom.Ny, geom.N), "e_in")
    if out is None:
        out = torch.empty((geom.L, geom.Py, geom.P), dtype=torch.float32, device=h.device)
    op = _dev_ptr(out, torch.float32, (geom.L, geom.Py, geom.P), "out")
    g = geom.c()
    need = int(L.load().doe_workspace_bytes(ctypes.byref(g), L.DOE_OP_PSF))
    ws, wp, wb = _ws_args(ws, need, h.device)
    L.check(L.load().doe_psf(ctypes.byref(g), hp, ep, op, wp, wb, _stream(stream)), "doe_psf")
    return out


def propagate(h: torch.Tensor, geom: Geometry, e_in: torch.Tensor | None = None, out: torch.Tensor | None = None,
              ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Destination fields E_dest (Eq. 3): complex64 [L, Py, Px]."""
    hp = _dev_ptr(h, torch.float32, (geom.NLy, geom.NL), "h")
    ep = _dev_ptr(e_in, torch.complex64, (geom.Ny, geom.N), "e_in")
    if out is None:
        out = torch.empty((geom.L, geom.Py, geom.P), dtype=torch.complex64, device=h.device)
    op = _dev_ptr(out, torch.complex64, (geom.L, geom.Py, geom.P), "out")
    g = geom.c()
    need = int(L.load().doe_workspace_bytes(ctypes.byref(g), L.DOE_OP_PROPAGATE))
    ws, wp, wb = _ws_args(ws, need, h.device)
    L.check(L.load().doe_propagate(ctypes.byref(g), hp, ep, op, wp, wb, _stream(stream)), "doe_propagate")
    return out


def psf_many(hs, geoms, e_ins=None, outs=None, ws: torch.Tensor | None = None, stream=None):
    """PSFs of several DOEs (same N and pad) in one set of launches."""
    n = len(geoms)
    gs = (L.Geom * n)(*[g.c() for g in geoms])
    if outs is None:
        outs = [torch.empty((g.L, g.Py, g.P), dtype=torch.float32, device=hs[0].device) for g in geoms]
    hp = (ctypes.c_void_p * n)(*[_dev_ptr(h, torch.float32, (g.NLy, g.NL), "h").value for h, g in zip(hs, geoms)])
    ep = (ctypes.c_void_p * n)(*[(e.data_ptr() if e is not None else None) for e in (e_ins or [None] * n)])
    op = (ctypes.c_void_p * n)(*[_dev_ptr(o, torch.float32, (g.L, g.Py, g.P), "out").value for o, g in zip(outs, geoms)])
    need = int(L.load().doe_workspace_bytes_many(n, gs, L.DOE_OP_PSF))
    ws, wp, wb = _ws_args(ws, need, hs[0].device)
    L.check(L.load().doe_psf_many(n, gs, hp, ep, op, wp, wb, _stream(stream)), "doe_psf_many")
    return outs


def grad(h: torch.Tensor, geom: Geometry, t_or_dldi: torch.Tensor, mode: str = "l2",
         e_in: torch.Tensor | None = None, recompute: bool = True, out: torch.Tensor | None = None,
         loss: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """(dL/dh float32 [Ny, N], loss float64 [1]) for L = sum (I - T)^2 (mode 'l2') or the
    vector-Jacobian product with dL/dI (mode 'vjp'; loss is then 0)."""
    hp = _dev_ptr(h, torch.float32, (geom.NLy, geom.NL), "h")
    ep = _dev_ptr(e_in, torch.complex64, (geom.Ny, geom.N), "e_in")
    tp = _dev_ptr(t_or_dldi, torch.float32, (geom.L, geom.Py, geom.P), "t_or_dldi")
    if out is None:
        out = torch.empty((geom.NLy, geom.NL), dtype=torch.float32, device=h.device)
    gp = _dev_ptr(out, torch.float32, (geom.NLy, geom.NL), "grad")
    if loss is None:
        loss = torch.empty((1,), dtype=torch.float64, device=h.device)
    lp = _dev_ptr(loss, torch.float64, (1,), "loss")
    g = geom.c()
    need = int(L.load().doe_workspace_bytes(ctypes.byref(g), L.DOE_OP_GRAD))
    ws, wp, wb = _ws_args(ws, need, h.device)
    m = L.DOE_GRAD_L2_TARGET if mode == "l2" else L.DOE_GRAD_VJP
    L.check(L.load().doe_grad(ctypes.byref(g), hp, ep, tp, m, gp, lp, int(bool(recompute)), wp, wb, _stream(stream)),
            "doe_grad")
    return out, loss


def render(psf_t: torch.Tensor, img: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Convolution of each image channel with its PSF (cropped at the axis, normalised)."""
    C, H, W = img.shape
    Py, Px = psf_t.shape[-2:]
    pp = _dev_ptr(psf_t, torch.float32, (C, Py, Px), "psf")
    ip = _dev_ptr(img, torch.float32, (C, H, W), "img")
    if out is None:
        out = torch.empty((C, H, W), dtype=torch.float32, device=img.device)
    op = _dev_ptr(out, torch.float32, (C, H, W), "out")
    need = int(L.load().doe_render_workspace_bytes(C, H, W))
    ws, wp, wb = _ws_args(ws, need, img.device)
    L.check(L.load().doe_render(C, H, W, pp, Py, Px, ip, op, wp, wb, _stream(stream)), "doe_render")
    return out


def wiener(psf_t: torch.Tensor, y: torch.Tensor, gamma: float, out: torch.Tensor | None = None,
           ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Wiener deconvolution of each blurred channel with its PSF (Eq. 9; crop at the axis,
    normalised, circular model)."""
    C, H, W = y.shape
    Py, Px = psf_t.shape[-2:]
    pp = _dev_ptr(psf_t, torch.float32, (C, Py, Px), "psf")
    yp = _dev_ptr(y, torch.float32, (C, H, W), "y")
    if out is None:
        out = torch.empty((C, H, W), dtype=torch.float32, device=y.device)
    op = _dev_ptr(out, torch.float32, (C, H, W), "out")
    need = int(L.load().doe_wiener_workspace_bytes(C, H, W))
    ws, wp, wb = _ws_args(ws, need, y.device)
    L.check(L.load().doe_wiener(C, H, W, pp, Py, Px, yp, float(gamma), op, wp, wb, _stream(stream)), "doe_wiener")
    return out


def radial_heights(c: torch.Tensor, n: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Radially symmetric heights [n][n] = sum_k c[k] s^k, s = (rho / R)^2 (c: float32 [n_c] on
    the device, n_c <= 9)."""
    n_c = c.numel()
    cp = _dev_ptr(c, torch.float32, (n_c,), "c")
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device=c.device)
    op = _dev_ptr(out, torch.float32, (n, n), "out")
    L.check(L.load().doe_radial_heights(int(n), cp, n_c, op, _stream(stream)), "doe_radial_heights")
    return out


def radial_grad(grad_h: torch.Tensor, n_c: int, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Coefficient gradient [n_c] = sum over the grid of grad_h * s^k (transpose of radial_heights)."""
    n = grad_h.shape[0]
    gp = _dev_ptr(grad_h, torch.float32, (n, n), "grad_h")
    if out is None:
        out = torch.empty((n_c,), dtype=torch.float32, device=grad_h.device)
    op = _dev_ptr(out, torch.float32, (n_c,), "out")
    need = int(L.load().doe_radial_workspace_bytes(int(n_c)))
    ws, wp, wb = _ws_args(ws, need, grad_h.device)
    L.check(L.load().doe_radial_grad(int(n), int(n_c), gp, op, wp, wb, _stream(stream)), "doe_radial_grad")
    return out


def adam_step(h: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, t: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, h_min: float = 0.0,
              h_max: float = float("inf"), stream=None) -> torch.Tensor:
    """One Adam step (step number t >= 1) on the heights h in place, then h clamped to
    [h_min, h_max]; m and v are the optimiser state (zeros before t = 1)."""
    n = h.numel()
    ptrs = [_dev_ptr(x, torch.float32, tuple(h.shape), name) for x, name in ((h, "h"), (grad, "grad"), (m, "m"), (v, "v"))]
    L.check(L.load().doe_adam_step(*ptrs, n, float(lr), float(beta1), float(beta2), float(eps), int(t), float(h_min),
                                   float(h_max), _stream(stream)), "doe_adam_step")
    return h


def band_limits(geom: Geometry):
    """(kmax [L] int32, m_ev [L] int64): the integer band logic the kernels apply."""
    k = np.zeros(geom.L, np.int32)
    m = np.zeros(geom.L, np.int64)
    g = geom.c()
    L.check(L.load().doe_band_limits(ctypes.byref(g), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "doe_band_limits")
    return k, m


def band_limits_xy(geom: Geometry):
    """(kmax_x [L] int32, kmax_y [L] int32, m_ev [L] int64): the per-axis band logic (equal to
    band_limits' kmax on both axes of a square grid)."""
    kx = np.zeros(geom.L, np.int32)
    ky = np.zeros(geom.L, np.int32)
    m = np.zeros(geom.L, np.int64)
    g = geom.c()
    i32 = ctypes.POINTER(ctypes.c_int32)
    L.check(L.load().doe_band_limits_xy(ctypes.byref(g), kx.ctypes.data_as(i32), ky.ctypes.data_as(i32),
                                        m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "doe_band_limits_xy")
    return kx, ky, m


def debug_band_mask(geom: Geometry, j: int, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The band mask (1 where H is kept) of wavelength j on the padded grid: uint8 [Py, Px]."""
    mask = torch.empty((geom.Py, geom.P), dtype=torch.uint8, device="cuda")
    g = geom.c()
    need = int(L.load().doe_workspace_bytes(ctypes.byref(g), L.DOE_OP_PSF))
    ws, wp, wb = _ws_args(ws, need, "cuda")
    L.check(L.load().doe_debug_band_mask(ctypes.byref(g), j, ctypes.c_void_p(mask.data_ptr()), wp, wb, _stream(stream)),
            "doe_debug_band_mask")
    return mask


class PSF(torch.autograd.Function):
    """Differentiable h -> PSF [L, Py, Px].  Backward runs the library's adjoint kernels
    (conjugate transfer function) with recomputation: no field is stored between passes."""

    @staticmethod
    def forward(ctx, h: torch.Tensor, geom: Geometry, e_in=None):
        ctx.geom = geom
        ctx.save_for_backward(h, e_in) if e_in is not None else ctx.save_for_backward(h)
        return psf(h, geom, e_in)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        saved = ctx.saved_tensors
        h = saved[0]
        e_in = saved[1] if len(saved) > 1 else None
        g, _ = grad(h, ctx.geom, grad_out.contiguous().float(), mode="vjp", e_in=e_in, recompute=True)
        return g, None, None


def psf_autograd(h: torch.Tensor, geom: Geometry, e_in=None) -> torch.Tensor:
    return PSF.apply(h, geom, e_in)


# ---------------------------------------------------------------- tracing
def trace_enable(max_records: int) -> None:
    """Bracket each of the next max_records pass launches with CUDA events (0 disables)."""
    L.check(L.load().doe_trace_enable(int(max_records)), "doe_trace_enable")


def trace_read(max_records: int = 1 << 16) -> list[tuple[str, float]]:
    """(pass name, device ms) of the traced launches since the last read, in launch order."""
    ids = (ctypes.c_int * max_records)()
    ms = (ctypes.c_float * max_records)()
    n = L.load().doe_trace_read(max_records, ids, ms)
    if n < 0:
        raise L.DoeError(n, "doe_trace_read")
    lib = L.load()
    return [(lib.doe_pass_name(ids[i]).decode(), float(ms[i])) for i in range(n)]


def fault_status() -> int:
    """OR of the kernels' fault bits (DOE_FAULT_*) since the last call, then cleared; 0 when
    every bounded wait completed and (in a DOE_DEBUG build) every index was in bounds."""
    w = ctypes.c_uint32(0)
    L.check(L.load().doe_fault_status(ctypes.byref(w)), "doe_fault_status")
    return int(w.value)


def debug_build() -> bool:
    return bool(L.load().doe_debug_build())


def check_wait_timeout(polls: int = 1 << 12, stream=None) -> None:
    """Launch the check of the bounded waits' failure path (a wait on a copy that is never
    issued); the next fault_status() reports DOE_FAULT_WAIT_TIMEOUT."""
    L.check(L.load().doe_check_wait_timeout(int(polls), _stream(stream)), "doe_check_wait_timeout")


def launch_count() -> int:
    """Number of kernels libdoe has launched in this process."""
    return int(L.load().doe_launch_count())
