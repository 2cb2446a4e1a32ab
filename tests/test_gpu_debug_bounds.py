"""The bounds-checked build (libdoe_debug.so, every kernel compiled with DOE_DEBUG): small
cases of every pass family run through its C ABI -- power-of-two grids (one CTA per transform),
split grids (32768 = 4 x 8192 and 65536 = 8 x 8192, the 16-CTA column clusters), mixed-radix
grids (one CTA; split over a cluster), rectangular grids, the adjoint passes, upsampled and
Lanczos layouts, incident fields, the circular band, render and Wiener.  In that build every global, shared and
distributed-shared-memory index is checked against its buffer before the access; the fault
word must stay 0, and the results must equal the release build's."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_22313_b300 import _lib as L
from paper_2505_22313_b300 import build, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    build.build()
    assert torch.cuda.is_available()
    rel, dbg = L.open_library(L.LIB_PATH), L.open_library(L.DEBUG_LIB_PATH)
    assert dbg.doe_debug_build() == 1 and rel.doe_debug_build() == 0
    return rel, dbg


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ws(lib, g, op):
    gc = g.c()
    n = int(lib.doe_workspace_bytes(ctypes.byref(gc), op))
    return torch.empty(max(n, 256), dtype=torch.uint8, device="cuda"), n


def _psf(lib, g, h, e_in=None, field=False):
    ws, n = _ws(lib, g, L.DOE_OP_PROPAGATE if field else L.DOE_OP_PSF)
    out = torch.full((g.L, g.Py, g.P) + ((2,) if field else ()), float("nan"), dtype=torch.float32, device="cuda")
    gc = g.c()
    fn = lib.doe_propagate if field else lib.doe_psf
    assert fn(ctypes.byref(gc), _p(h), _p(e_in), _p(out), _p(ws), n, _stream()) == L.DOE_OK
    return out


def _grad(lib, g, h, T, e_in=None):
    ws, n = _ws(lib, g, L.DOE_OP_GRAD)
    gr = torch.full((g.NLy, g.NL), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    gc = g.c()
    assert lib.doe_grad(ctypes.byref(gc), _p(h), _p(e_in), _p(T), L.DOE_GRAD_L2_TARGET, _p(gr), _p(loss), 1, _p(ws), n,
                        _stream()) == L.DOE_OK
    return gr, loss


def _faults(lib):
    w = ctypes.c_uint32(0xFFFFFFFF)
    assert lib.doe_fault_status(ctypes.byref(w)) == L.DOE_OK
    return int(w.value)


def _same(a, b, tol=1e-6):
    a, b = a.double(), b.double()
    assert torch.isfinite(a).all()
    err = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
    assert err <= tol, err


CASES = [
    # (name, N, pad, dx, z, wavelengths, keyword arguments of Geometry.make, gradient)
    ("pow2", 128, 2, 1e-6, 2e-3, [450e-9, 633e-9], {}, True),
    ("pow2_pad1", 256, 1, 1e-6, 1e-3, [550e-9], {}, True),
    ("pow2_8192", 4096, 2, 1e-6, 50e-3, [550e-9], {}, True),
    ("pow2_16384", 8192, 2, 1e-6, 50e-3, [650e-9], {}, False),
    ("tilt_sphere_upsampled", 256, 2, 1e-6, 5e-3, [500e-9], dict(upsample=2, theta_x=0.01, src_d=-0.05), True),
    ("lanczos", 256, 2, 1e-6, 5e-3, [520e-9], dict(upsample=4, lanczos=True), True),
    ("circular", 256, 2, 2e-6, 20e-3, [550e-9], dict(bandlimit="circular"), True),
    ("kmax0", 128, 2, 1e-6, 0.1, [550e-9], {}, True),  # one stored column pair, a 2-entry H row
    ("kmax0_mixed", 90, 2, 1e-6, 0.1, [550e-9], {}, True),
    ("mixed_radix", 180, 2, 1e-6, 2e-3, [450e-9, 600e-9], {}, True),
    ("mixed_radix_split", 4500, 2, 1e-6, 5e-3, [550e-9], {}, True),
    ("mixed_radix_split_pairs", 9000, 2, 1e-6, 5e-3, [550e-9], {}, True),  # 18000 = 8 x 2250: two columns per 16-CTA cluster
    ("split_32768", 16384, 2, 1e-6, 50e-3, [550e-9], {}, True),
    ("split_65536", 32768, 2, 1e-6, 100e-3, [550e-9], {}, False),
    ("rect_mixed", 160, 2, 1e-6, 2e-3, [450e-9, 600e-9], dict(Ny=96), True),
    ("rect_pow2_pad1", 256, 1, 1e-6, 2e-3, [550e-9], dict(Ny=512), True),
    ("rect_large", 4000, 2, 1e-6, 20e-3, [550e-9], dict(Ny=3000), True),
    ("rect_split_rows", 4500, 2, 1e-6, 10e-3, [550e-9], dict(Ny=500), True),      # Px = 9000 = 8 x 1125
    ("rect_split_cols_pairs", 300, 2, 1e-6, 10e-3, [550e-9], dict(Ny=9000), True),  # Py = 18000 = 8 x 2250
    ("rect_split16_rows", 64320, 2, 1e-6, 20e-3, [550e-9], dict(Ny=100), True),  # Px = 128640 = 16 x 8040
]


@pytest.mark.parametrize("name,N,pad,dx,z,lams,kw,grad", CASES, ids=[c[0] for c in CASES])
def test_bounds_checked_build_matches_release(libs, name, N, pad, dx, z, lams, kw, grad):
    rel, dbg = libs
    g = Geometry.make(N, dx, z, lams, pad=pad, **kw)
    nl = g.NL
    if g.Ny != N and max(N, g.Ny) > 16384:  # a long thin rectangle: uniform random heights
        h = torch.from_numpy(np.random.default_rng(4000 + N).random((g.Ny, N), dtype=np.float32) * np.float32(1.2e-6)).cuda()
    elif g.Ny != N:  # rectangle: the top-left Ny x N block of a square map
        h = torch.from_numpy(np.ascontiguousarray(inputs.heights(max(N, g.Ny), 4000 + N)[:g.Ny, :N])).cuda()
    elif nl <= 8192:
        h = torch.from_numpy(inputs.heights(nl, 4000 + N)).cuda()
    else:
        h = inputs.heights_device(nl, 4000 + N, "cuda")
    e_in = None
    if name == "pow2":
        rng = np.random.default_rng(1)
        e_in = torch.from_numpy((rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)).cuda()
    _faults(dbg)  # clear
    a = _psf(dbg, g, h, e_in)
    assert _faults(dbg) == 0
    _same(a, _psf(rel, g, h, e_in))
    del a
    if name in ("pow2", "mixed_radix", "rect_mixed"):
        f = _psf(dbg, g, h, e_in, field=True)
        assert _faults(dbg) == 0
        _same(f, _psf(rel, g, h, e_in, field=True))
    if grad:
        if max(g.P, g.Py) > 32768:  # long thin rectangle: a uniform random target of the grid's shape
            gen = torch.Generator(device="cuda").manual_seed(5000 + N)
            T = torch.rand((g.L, g.Py, g.P), generator=gen, device="cuda") * (N * g.Ny / (g.P * g.Py))
        else:
            T = inputs.spot_target_device(max(g.P, g.Py), max(N, g.Ny), g.L, 5000 + N, "cuda")[:, :g.Py, :g.P].contiguous()
        gd, ld = _grad(dbg, g, h, T, e_in)
        assert _faults(dbg) == 0
        gr, lr = _grad(rel, g, h, T, e_in)
        _same(gd, gr, 1e-5)
        _same(ld, lr, 1e-9)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _render(lib, fn, C, H, W, psf, img, gamma=None):
    ws_n = int((lib.doe_wiener_workspace_bytes if gamma is not None else lib.doe_render_workspace_bytes)(C, H, W))
    ws = torch.empty(ws_n, dtype=torch.uint8, device="cuda")
    out = torch.full((C, H, W), float("nan"), dtype=torch.float32, device="cuda")
    Py, Px = psf.shape[1], psf.shape[2]
    if gamma is None:
        rc = lib.doe_render(C, H, W, _p(psf), Py, Px, _p(img), _p(out), _p(ws), ws_n, _stream())
    else:
        rc = lib.doe_wiener(C, H, W, _p(psf), Py, Px, _p(img), ctypes.c_double(gamma), _p(out), _p(ws), ws_n, _stream())
    assert rc == L.DOE_OK
    return out


@pytest.mark.parametrize("C,H,W,Pp", [(3, 256, 256, 512), (2, 64, 128, 256)])
def test_bounds_checked_render_and_wiener(libs, C, H, W, Pp):
    rel, dbg = libs
    rng = np.random.default_rng(7)
    psf = torch.from_numpy(rng.random((C, Pp, Pp), dtype=np.float32) ** 4).cuda()
    img = torch.from_numpy(inputs.image(C, H, W, 2100)).cuda()
    _faults(dbg)
    for gamma in (None, 5e-4):
        a = _render(dbg, None, C, H, W, psf, img, gamma)
        assert _faults(dbg) == 0
        _same(a, _render(rel, None, C, H, W, psf, img, gamma))
