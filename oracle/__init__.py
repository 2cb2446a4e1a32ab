"""FP64 CPU oracle for the DOE scalar-diffraction path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never does, and this package imports nothing
from it: the two share no code.  The propagation, PSF, gradient and render arithmetic lives in
``doe_oracle.c`` (plain C, FP64, its own FFT for any length); this module compiles it, marshals
numpy arrays, and writes out in FP64 numpy the smaller definitions (incident fields,
upsampling, the radial parameterisation, Adam) and the rectangular-grid propagation (on the
C oracle's 2-D FFT, which takes ny != nx).

Every function follows Wei et al., "Large-Area Fabrication-Aware Computational Diffractive
Optics" (TOG 2025), Sec. 3.1:
  * Eq. 1  phase  Phi = 2 pi (n - 1) h / lambda
  * Eq. 2  field  E_doe = E_in exp(+i Phi)
  * Eq. 3  angular-spectrum propagation with the band-limited transfer function H
  * I = |E_dest|^2 (PSF), and the gradient of Eq. 4's objective with an L2 penalty.
Parity is pinned in ``tests/test_oracle_pins.py`` against closed forms, invariants, brute
force and a Rayleigh-Sommerfeld direct sum; no pin compares the oracle with itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "doe_oracle.c"
_LIB_PATH = _HERE / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile doe_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.run(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(tmp), str(_SRC), "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    P = ctypes.c_void_p
    L = ctypes.c_long
    D = ctypes.c_double
    Ii = ctypes.c_int
    sig = {
        "orc_num_threads": ([], Ii),
        "orc_fft1d": ([P, L, Ii], None),
        "orc_fft2d": ([P, L, L, Ii], Ii),
        "orc_dft1d": ([P, P, L, Ii], None),
        "orc_kmax": ([D, D, L, D, Ii], L),
        "orc_mev": ([D, D, L], ctypes.c_int64),
        "orc_mlim": ([D, D, L, D, Ii], ctypes.c_int64),
        "orc_transfer": ([P, L, D, D, D, Ii], None),
        "orc_band_mask": ([P, L, D, D, D, Ii], None),
        "orc_propagate": ([L, L, D, D, D, D, Ii, P, P, P], Ii),
        "orc_psf": ([L, L, D, D, D, D, Ii, P, P, P], Ii),
        "orc_psf_rows": ([L, L, D, D, D, D, Ii, P, P, L, P, P], Ii),
        "orc_grad_rows": ([L, L, D, D, D, D, Ii, P, P, L, P, P, L, P, P], Ii),
        "orc_grad": ([L, L, D, D, L, P, P, Ii, P, P, P, Ii, P, P], Ii),
        "orc_loss_l2": ([L, L, D, D, L, P, P, Ii, P, P, P, P], Ii),
        "orc_fd_exact": ([L, L, D, D, L, P, P, Ii, P, P, P, L, P, P, D, P], Ii),
        "orc_render": ([L, L, L, P, L, L, P, P], Ii),
        "orc_wiener": ([L, L, L, P, L, L, P, D, P], Ii),
        "orc_rs_direct": ([L, L, D, D, D, P, P], Ii),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c128(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _bl(bandlimit) -> int:
    """Band-limit mode of the C oracle: 0 none, 1 the separable square (the default reading),
    2 the circular disc (bandlimit="circular")."""
    if isinstance(bandlimit, str):
        if bandlimit != "circular":
            raise ValueError(f"unknown band limit {bandlimit!r}")
        return 2
    return int(bool(bandlimit))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- FFT
def fft(x, inverse: bool = False) -> np.ndarray:
    """Unnormalised 1-D DFT (sign -1 forward, +1 inverse) with the oracle's FFT (any length)."""
    a = np.array(x, dtype=np.complex128, copy=True)
    _load().orc_fft1d(_ptr(a), a.shape[0], +1 if inverse else -1)
    return a


def fft2(x, inverse: bool = False) -> np.ndarray:
    a = np.array(x, dtype=np.complex128, copy=True)
    _check(_load().orc_fft2d(_ptr(a), a.shape[0], a.shape[1], +1 if inverse else -1), "fft2")
    return a


def dft(x, inverse: bool = False) -> np.ndarray:
    """Plain O(n^2) DFT (brute force)."""
    a = _c128(x)
    out = np.empty_like(a)
    _load().orc_dft1d(_ptr(a), _ptr(out), a.shape[0], +1 if inverse else -1)
    return out


# ---------------------------------------------------------------- band limit / H
def kmax(lam: float, dx: float, P: int, z: float, bandlimit: bool = True) -> int:
    return int(_load().orc_kmax(lam, dx, P, z, _bl(bandlimit)))


def m_ev(lam: float, dx: float, P: int) -> int:
    return int(_load().orc_mev(lam, dx, P))


def m_lim(lam: float, dx: float, P: int, z: float, bandlimit=True) -> int:
    """The bound of m = kt^2 + lt^2 the transfer function applies: the evanescent m_ev, and
    for the circular band limit min(m_ev, ceil((f_lim / du)^2))."""
    return int(_load().orc_mlim(lam, dx, P, z, _bl(bandlimit)))


def transfer(P: int, dx: float, z: float, lam: float, bandlimit: bool = True) -> np.ndarray:
    H = np.empty((P, P), np.complex128)
    _load().orc_transfer(_ptr(H), P, dx, z, lam, _bl(bandlimit))
    return H


def band_mask(P: int, dx: float, z: float, lam: float, bandlimit: bool = True) -> np.ndarray:
    m = np.empty((P, P), np.uint8)
    _load().orc_band_mask(_ptr(m), P, dx, z, lam, _bl(bandlimit))
    return m


# ---------------------------------------------------------------- forward path
def propagate(h, dx, z, lam, n_index=1.46, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """E_dest on the P x P grid for one wavelength (Eq. 1-3)."""
    h = _f32(h)
    N = h.shape[0]
    P = pad * N
    out = np.empty((P, P), np.complex128)
    e_in = _c128(e_in)
    _check(
        _load().orc_propagate(N, pad, dx, z, lam, n_index, _bl(bandlimit), _ptr(h), _ptr(e_in), _ptr(out)),
        "propagate",
    )
    return out


def psf(h, dx, z, lams, n_index=None, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """FP64 PSFs [L][P][P] = |E_dest|^2 per wavelength."""
    h = _f32(h)
    lams = np.atleast_1d(np.asarray(lams, np.float64))
    nidx = np.full(lams.shape, 1.46) if n_index is None else np.broadcast_to(np.asarray(n_index, np.float64), lams.shape)
    N = h.shape[0]
    P = pad * N
    out = np.empty((lams.size, P, P), np.float64)
    e_in = _c128(e_in)
    for j, lam in enumerate(lams):
        _check(
            _load().orc_psf(N, pad, dx, z, float(lam), float(nidx[j]), _bl(bandlimit), _ptr(h), _ptr(e_in), _ptr(out[j])),
            "psf",
        )
    return out


def psf_rows(h, dx, z, lam, rows, n_index=1.46, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """Exact FP64 PSF rows ``rows`` of one wavelength without holding the P x P field."""
    h = _f32(h)
    N = h.shape[0]
    P = pad * N
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.size, P), np.float64)
    e_in = _c128(e_in)
    _check(
        _load().orc_psf_rows(N, pad, dx, z, lam, n_index, _bl(bandlimit), _ptr(h), _ptr(e_in), rows.size, _ptr(rows), _ptr(out)),
        "psf_rows",
    )
    return out


# ---------------------------------------------------------------- rectangular grids
# Sides Py x Px (Table 2's 128640 x 85760 large-area grid is not square), transformed with the
# oracle's own FFT.  Reading of Sec. 3.1 for Py != Px: each axis keeps its own frequency step
# (dux = 1 / (Px dx), duy = 1 / (Py dx)) and its own band limit (the square rule per axis:
# kmax_x = ceil(flim_x / dux) - 1 capped at Px / 2 with flim_x = 1 / (lambda sqrt((2 dux z)^2
# + 1)), likewise in y); a sample propagates iff lambda^2 (fx^2 + fy^2) < 1.  With g = gcd(Px,
# Py), A = Px / g, B = Py / g that is the integer rule kx^2 B^2 + ky^2 A^2 < M_ev,
# M_ev = ceil((Px Py dx / (g lambda))^2) evaluated once in FP64 (exact integers on the left).
def _kmax_axis(lam: float, dx: float, P: int, z: float, bandlimit: bool) -> int:
    if isinstance(bandlimit, str):
        raise ValueError("rectangular grids take the separable band limit only")
    if not bandlimit:
        return P // 2
    du = 1.0 / (P * dx)
    flim = 1.0 / (lam * np.sqrt((2.0 * du * z) ** 2 + 1.0))
    return int(min(max(np.ceil(flim / du) - 1, 0), P // 2))


def mev_rect(Py: int, Px: int, dx: float, lam: float) -> tuple[int, int, int]:
    """(A^2, B^2, M_ev) of the rectangular evanescent rule kx^2 B^2 + ky^2 A^2 < M_ev."""
    g = int(np.gcd(Px, Py))
    a, b = Px // g, Py // g
    x = float(Px) * float(Py) * dx / (float(g) * lam)
    return a * a, b * b, int(np.ceil(x * x))


def kmax_rect(Py: int, Px: int, dx: float, z: float, lam: float, bandlimit: bool = True) -> tuple[int, int]:
    """(kmax_x, kmax_y) of a rectangular grid."""
    return _kmax_axis(lam, dx, Px, z, bandlimit), _kmax_axis(lam, dx, Py, z, bandlimit)


def band_mask_rect(Py: int, Px: int, dx: float, z: float, lam: float, bandlimit: bool = True) -> np.ndarray:
    """[Py][Px] uint8 band mask (1 = H != 0) of a rectangular grid, FFT order."""
    kx = np.where(np.arange(Px) < Px // 2, np.arange(Px), np.arange(Px) - Px).astype(np.int64)
    ky = np.where(np.arange(Py) < Py // 2, np.arange(Py), np.arange(Py) - Py).astype(np.int64)
    a2, b2, mev = mev_rect(Py, Px, dx, lam)
    kxm, kym = kmax_rect(Py, Px, dx, z, lam, bandlimit)
    m = kx[None, :] ** 2 * b2 + ky[:, None] ** 2 * a2
    return ((np.abs(kx)[None, :] <= kxm) & (np.abs(ky)[:, None] <= kym) & (m < mev)).astype(np.uint8)


def transfer_rect(Py: int, Px: int, dx: float, z: float, lam: float, bandlimit: bool = True) -> np.ndarray:
    """[Py][Px] complex128 band-limited transfer function, FFT order, Nyquist at -P/2."""
    kx = np.where(np.arange(Px) < Px // 2, np.arange(Px), np.arange(Px) - Px).astype(np.float64)
    ky = np.where(np.arange(Py) < Py // 2, np.arange(Py), np.arange(Py) - Py).astype(np.float64)
    fx = kx / (Px * dx)
    fy = ky / (Py * dx)
    band = band_mask_rect(Py, Px, dx, z, lam, bandlimit).astype(bool)
    H = np.zeros((Py, Px), np.complex128)
    H[band] = np.exp(2j * np.pi * z * np.sqrt(1.0 / (lam * lam) - (fx[None, :] ** 2 + fy[:, None] ** 2)[band]))
    return H


def _fft2r(a):
    return fft2(a)


def _ifft2r(a):
    return fft2(a, inverse=True) / (a.shape[0] * a.shape[1])


def _doe_field_rect(h, lam, n_index, e_in):
    h = np.asarray(h)
    h64 = h if h.dtype == np.float64 else h.astype(np.float32).astype(np.float64)  # float64 kept as is (FD)
    e = np.exp(1j * 2 * np.pi * (n_index - 1.0) * h64 / lam)
    return e if e_in is None else e * np.asarray(e_in, np.complex128)


def propagate_rect(h, dx, z, lam, n_index=1.46, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """E_dest [pad Ny][pad Nx] for heights [Ny][Nx] (Eq. 1-3), DOE at offset ((P - N) / 2) per axis."""
    Ny, Nx = np.asarray(h).shape
    Py, Px = pad * Ny, pad * Nx
    E = np.zeros((Py, Px), np.complex128)
    E[(Py - Ny) // 2:(Py - Ny) // 2 + Ny, (Px - Nx) // 2:(Px - Nx) // 2 + Nx] = _doe_field_rect(h, lam, n_index, e_in)
    return _ifft2r(_fft2r(E) * transfer_rect(Py, Px, dx, z, lam, bandlimit))


def psf_rect(h, dx, z, lams, n_index=1.46, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """FP64 PSFs [L][Py][Px] on a rectangular grid."""
    return np.stack([np.abs(propagate_rect(h, dx, z, lam, n_index, pad, e_in, bandlimit)) ** 2
                     for lam in np.atleast_1d(lams)])


def grad_rect(h, dx, z, lams, target, n_index=1.46, pad=2, e_in=None, bandlimit=True):
    """(dL/dh [Ny][Nx], L) for L = sum_lambda sum (I - T)^2 on a rectangular grid: g_out = 2 (I - T) E,
    g_pad = IFFT2(conj(H) FFT2(g_out)), dL/dh = sum_lambda -2 k' Im(conj(g_doe) E_doe)."""
    Ny, Nx = np.asarray(h).shape
    Py, Px = pad * Ny, pad * Nx
    oy, ox = (Py - Ny) // 2, (Px - Nx) // 2
    g = np.zeros((Ny, Nx))
    loss = 0.0
    for j, lam in enumerate(np.atleast_1d(lams)):
        H = transfer_rect(Py, Px, dx, z, lam, bandlimit)
        ed = _doe_field_rect(h, lam, n_index, e_in)
        E = np.zeros((Py, Px), np.complex128)
        E[oy:oy + Ny, ox:ox + Nx] = ed
        Eo = _ifft2r(_fft2r(E) * H)
        d = np.abs(Eo) ** 2 - np.asarray(target[j], np.float64)
        loss += float((d * d).sum())
        gp = _ifft2r(np.conj(H) * _fft2r(2.0 * d * Eo))[oy:oy + Ny, ox:ox + Nx]
        kp = 2 * np.pi * (n_index - 1.0) / lam
        g += -2.0 * kp * np.imag(np.conj(gp) * ed)
    return g, loss


# ---------------------------------------------------------------- incident fields
def incident(N: int, dx: float, lam: float, theta_x: float = 0.0, theta_y: float = 0.0, d: float = 0.0) -> np.ndarray:
    """E_in [N][N] complex128 of Eq. 2 for a plane or spherical incident wave (Sec. 3.1 names
    both; Sec. 2.3 scales over incidence angles), read as: sample (i, j) at x = (j - N/2) dx,
    y = (i - N/2) dx (the optical axis at padded index P/2);
        tilt:   exp(+i 2 pi (x sin theta_x + y sin theta_y) / lambda)
        sphere: 1 if d == 0, else (|d| / r) exp(+i sgn(d) 2 pi (r - |d|) / lambda),
                r = sqrt(x^2 + y^2 + d^2)
    and E_in = tilt * sphere.  d > 0 is a point source |d| before the DOE (diverging wave),
    d < 0 a wave converging to the point |d| behind it; phases are referenced to the axis."""
    c = (np.arange(N, dtype=np.float64) - N // 2) * dx
    y = c[:, None]
    x = c[None, :]
    e = np.exp(2j * np.pi * (x * np.sin(theta_x) + y * np.sin(theta_y)) / lam)
    if d != 0.0:
        r = np.sqrt(x * x + y * y + d * d)
        e = e * (abs(d) / r) * np.exp(1j * np.sign(d) * 2 * np.pi * (r - abs(d)) / lam)
    return e


# ---------------------------------------------------------------- radial parameterisation
def radial_s(N: int) -> np.ndarray:
    """[N][N] squared normalised radius s = rho^2 / R^2 of each sample, rho measured from the
    optical axis at sample (N/2, N/2) and R = N dx / 2 the half-aperture (dx cancels)."""
    c = np.arange(N, dtype=np.float64) - N // 2
    return (c[:, None] ** 2 + c[None, :] ** 2) / (N / 2.0) ** 2


def radial_heights(c, N: int) -> np.ndarray:
    """Radially symmetric height map of Sec. 5.4's broadband design (radial symmetry through a
    16th-order polynomial), read as an even polynomial in rho / R:
    h = sum_k c[k] s^k, s = (rho / R)^2, k = 0 .. len(c) - 1 <= 8 (degree <= 16).  FP64."""
    c = np.asarray(c, np.float64)
    s = radial_s(N)
    return sum(ck * s**k for k, ck in enumerate(c))


def radial_grad(g, n_c: int) -> np.ndarray:
    """dL/dc[k] = sum over the grid of dL/dh * s^k (the transpose of radial_heights). FP64."""
    g = np.asarray(g, np.float64)
    s = radial_s(g.shape[0])
    return np.array([(g * s**k).sum() for k in range(n_c)])


# ---------------------------------------------------------------- design optimiser
def adam_step(h, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, h_min=0.0, h_max=np.inf):
    """One Adam step (Kingma & Ba 2015, the optimiser of the paper's designs, Sec. 3.2) in FP64,
    then projection onto [h_min, h_max]; returns (h, m, v)."""
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1**t)
    v_hat = v / (1.0 - beta2**t)
    h = np.asarray(h, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return np.clip(h, h_min, h_max), m, v


def cosine_lr(lr0, t, iters):
    """Cosine decay of the learning rate to zero over iters steps (Sec. 3.2's schedule), t = 1.."""
    return 0.5 * lr0 * (1.0 + np.cos(np.pi * (t - 1) / iters))


# ---------------------------------------------------------------- super-resolved design input
def upsample_nearest(h_layout, f: int) -> np.ndarray:
    """Heights on the simulation grid from a layout at f times its pitch by nearest (zero-order)
    upsampling, the interpolation the paper's conventional large-area designs use (Sec. 3.2, toy
    example; Sec. 5.2: 8x and 4x nearest upsampling): h[i][x] = h_layout[i // f][x // f]."""
    return np.repeat(np.repeat(np.asarray(h_layout, np.float32), f, axis=0), f, axis=1)


def layout_grad(g_sim, f: int) -> np.ndarray:
    """Gradient on the layout from the gradient on the simulation grid: the adjoint of
    upsample_nearest, i.e. the sum over each f x f block."""
    g = np.asarray(g_sim, np.float64)
    n = g.shape[0] // f
    return g.reshape(n, f, n, f).sum(axis=(1, 3))


def lanczos3_matrix(n_layout: int, f: int) -> np.ndarray:
    """[n_layout f][n_layout] FP64 interpolation matrix of Lanczos-3 upsampling by f, the
    smooth kernel the paper compares nearest upsampling against (Sec. 3.2, toy example), read
    as: sample x at layout coordinate u = (x + 1/2) / f - 1/2 (cell centres), weights
    K(u - n) = sinc(u - n) sinc((u - n) / 3) for |u - n| < 3 normalised to sum 1, cells
    clamped to the layout at its edges."""
    n = n_layout * f
    W = np.zeros((n, n_layout))
    for x in range(n):
        u = (x + 0.5) / f - 0.5
        taps = np.arange(int(np.floor(u)) - 2, int(np.floor(u)) + 4)
        t = u - taps
        k = np.where(np.abs(t) < 3.0, np.sinc(t) * np.sinc(t / 3.0), 0.0)
        k /= k.sum()
        for tap, wgt in zip(taps, k):
            W[x, min(max(tap, 0), n_layout - 1)] += wgt
    return W


def upsample_lanczos3(h_layout, f: int) -> np.ndarray:
    """Heights on the simulation grid from the layout by separable Lanczos-3 interpolation."""
    hl = np.asarray(h_layout, np.float64)
    W = lanczos3_matrix(hl.shape[0], f)
    return (W @ hl @ W.T).astype(np.float32)


def layout_grad_lanczos3(g_sim, f: int) -> np.ndarray:
    """Layout gradient: the transpose of upsample_lanczos3 applied to the simulation-grid one."""
    g = np.asarray(g_sim, np.float64)
    W = lanczos3_matrix(g.shape[0] // f, f)
    return W.T @ g @ W


def grad_rows(h, dx, z, lam, rows, g_rows, drows, n_index=1.46, pad=2, e_in=None, bandlimit=True) -> np.ndarray:
    """Exact FP64 dL/dh on the DOE rows ``drows`` [len(drows)][N] for one wavelength, when
    dL/dI is ``g_rows`` [len(rows)][P] on the output rows ``rows`` (distinct) and zero on every
    other row, without holding the P x P field."""
    h = _f32(h)
    N = h.shape[0]
    P = pad * N
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    drows = np.ascontiguousarray(drows, dtype=np.int64)
    if np.unique(rows).size != rows.size:
        raise ValueError("rows must be distinct")
    g_rows = _f32(g_rows).reshape(rows.size, P)
    out = np.empty((drows.size, N), np.float64)
    e_in = _c128(e_in)
    _check(
        _load().orc_grad_rows(N, pad, dx, z, lam, n_index, _bl(bandlimit), _ptr(h), _ptr(e_in), rows.size, _ptr(rows),
                              _ptr(g_rows), drows.size, _ptr(drows), _ptr(out)),
        "grad_rows",
    )
    return out


def grad(h, dx, z, lams, t_or_g, n_index=None, pad=2, e_in=None, mode="l2", bandlimit=True):
    """(dL/dh [N][N] FP64, loss) for L = sum_j sum (I_j - T_j)^2 (mode 'l2') or the VJP
    with dL/dI = t_or_g (mode 'vjp'; loss is then 0)."""
    h = _f32(h)
    lams = np.atleast_1d(np.asarray(lams, np.float64))
    nidx = np.full(lams.shape, 1.46) if n_index is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n_index, np.float64), lams.shape))
    N = h.shape[0]
    P = pad * N
    t = _f32(t_or_g).reshape(lams.size, P, P)
    g = np.empty((N, N), np.float64)
    loss = ctypes.c_double(0.0)
    e_in = _c128(e_in)
    _check(
        _load().orc_grad(N, pad, dx, z, lams.size, _ptr(lams), _ptr(nidx), _bl(bandlimit), _ptr(h), _ptr(e_in),
                         _ptr(t), 0 if mode == "l2" else 1, _ptr(g), ctypes.byref(loss)),
        "grad",
    )
    return g, float(loss.value)


def loss_l2(h64, dx, z, lams, target, n_index=None, pad=2, e_in=None, bandlimit=True) -> float:
    h64 = np.ascontiguousarray(h64, np.float64)
    lams = np.atleast_1d(np.asarray(lams, np.float64))
    nidx = np.full(lams.shape, 1.46) if n_index is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n_index, np.float64), lams.shape))
    N = h64.shape[0]
    P = pad * N
    t = _f32(target).reshape(lams.size, P, P)
    out = ctypes.c_double(0.0)
    e_in = _c128(e_in)
    _check(
        _load().orc_loss_l2(N, pad, dx, z, lams.size, _ptr(lams), _ptr(nidx), _bl(bandlimit), _ptr(h64), _ptr(e_in), _ptr(t), ctypes.byref(out)),
        "loss",
    )
    return float(out.value)


def fd_exact(h, dx, z, lams, target, pix_y, pix_x, eps, n_index=None, pad=2, e_in=None, bandlimit=True):
    """Central finite differences of the L2 loss at the given DOE pixels, evaluated by exact
    FP64 differences (no cancellation)."""
    h = _f32(h)
    lams = np.atleast_1d(np.asarray(lams, np.float64))
    nidx = np.full(lams.shape, 1.46) if n_index is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n_index, np.float64), lams.shape))
    N = h.shape[0]
    P = pad * N
    t = _f32(target).reshape(lams.size, P, P)
    py = np.ascontiguousarray(pix_y, np.int64)
    px = np.ascontiguousarray(pix_x, np.int64)
    out = np.empty(py.size, np.float64)
    e_in = _c128(e_in)
    _check(
        _load().orc_fd_exact(N, pad, dx, z, lams.size, _ptr(lams), _ptr(nidx), _bl(bandlimit), _ptr(h), _ptr(e_in),
                             _ptr(t), py.size, _ptr(py), _ptr(px), eps, _ptr(out)),
        "fd_exact",
    )
    return out


# ---------------------------------------------------------------- render / wiener / RS
def render(psf_arr, img) -> np.ndarray:
    psf_arr = _f32(psf_arr)
    img = _f32(img)
    C, H, W = img.shape
    Py, Px = psf_arr.shape[-2:]
    out = np.empty((C, H, W), np.float64)
    _check(_load().orc_render(C, H, W, _ptr(psf_arr), Py, Px, _ptr(img), _ptr(out)), "render")
    return out


def wiener(psf_arr, y, gamma) -> np.ndarray:
    psf_arr = _f32(psf_arr)
    y = _f32(y)
    C, H, W = y.shape
    Py, Px = psf_arr.shape[-2:]
    out = np.empty((C, H, W), np.float64)
    _check(_load().orc_wiener(C, H, W, _ptr(psf_arr), Py, Px, _ptr(y), gamma, _ptr(out)), "wiener")
    return out


def rs_direct(e_doe, P, dx, z, lam) -> np.ndarray:
    e_doe = _c128(e_doe)
    N = e_doe.shape[0]
    out = np.empty((P, P), np.complex128)
    _check(_load().orc_rs_direct(N, P, dx, z, lam, _ptr(e_doe), _ptr(out)), "rs_direct")
    return out
