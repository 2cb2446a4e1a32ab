"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry
point include/doe.h declares, applies the band logic bit-exactly like the oracle, and
rejects bad arguments before launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2505_22313_b300 import _lib as L
from paper_2505_22313_b300 import build
from paper_2505_22313_b300.api import Geometry, band_limits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "doe.h")).read()
    declared = set(re.findall(r"^\s*(?:int|size_t|long long|const char\*)\s+(doe_\w+)\(", hdr, re.M))
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(L.EXPORTS) | {"doe_render_workspace_bytes"}


def test_binding_constants_match_header():
    # the Python binding's error codes and sizes are the header's #define values
    hdr = open(os.path.join(ROOT, "include", "doe.h")).read()
    defs = dict(re.findall(r"^#define\s+(DOE_\w+)\s+(.+?)\s*(?:/\*.*)?$", hdr, re.M))
    m = re.fullmatch(r"\((\d+)u?\s*<<\s*(\d+)\)", defs["DOE_NOALLOC_SCRATCH_BYTES"])
    assert m and L.DOE_NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))
    for name in ("DOE_OK", "DOE_EINVAL", "DOE_EUNSUPPORTED", "DOE_ENOWS", "DOE_ECUDA", "DOE_ETIMEDOUT", "DOE_ESCRATCH"):
        assert getattr(L, name) == int(defs[name].strip("()")), name


CASES = [
    (256, 2, 2e-6, 20e-3, [550e-9]),
    (4096, 2, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9]),
    (8192, 2, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9]),
    (32768, 2, 1e-6, 100e-3, [550e-9]),
    (64, 2, 0.25e-6, 5e-6, [400e-9, 700e-9]),
    (1024, 1, 1e-6, 10e-3, [520.6e-9]),
]


@pytest.mark.parametrize("N,pad,dx,z,lams", CASES)
def test_band_limits_bit_exact_vs_oracle(lib, N, pad, dx, z, lams):
    g = Geometry.make(N, dx, z, lams, pad=pad)
    k, m = band_limits(g)
    P = pad * N
    for j, lam in enumerate(lams):
        assert int(k[j]) == oracle.kmax(lam, dx, P, z)
        assert int(m[j]) == oracle.m_ev(lam, dx, P)


def test_band_limits_random_geometries(lib):
    rng = np.random.default_rng(99)
    for _ in range(200):
        N = int(2 ** rng.integers(4, 15))
        dx = float(rng.uniform(0.2e-6, 4e-6))
        z = float(10 ** rng.uniform(-5, -0.5))
        lam = float(rng.uniform(380e-9, 780e-9))
        g = Geometry.make(N, dx, z, [lam])
        k, m = band_limits(g)
        assert int(k[0]) == oracle.kmax(lam, dx, 2 * N, z)
        assert int(m[0]) == oracle.m_ev(lam, dx, 2 * N)
        # circular band: the same kmax, the bound of kt^2 + lt^2 including the disc
        kc, mc = band_limits(Geometry.make(N, dx, z, [lam], bandlimit="circular"))
        assert int(kc[0]) == int(k[0])
        assert int(mc[0]) == oracle.m_lim(lam, dx, 2 * N, z, "circular")


def _geom(**kw):
    base = dict(N=64, dx=1e-6, z=1e-3, lambdas=[550e-9])
    base.update(kw)
    return Geometry.make(**base)


def test_band_limits_rect_bit_exact_vs_oracle(lib):
    """Per-axis kmax and the rectangular evanescent bound M_ev (kx^2 B^2 + ky^2 A^2 < M_ev)
    equal the oracle's integers; on a square grid the x and y limits equal band_limits'."""
    from paper_2505_22313_b300.api import band_limits_xy
    rng = np.random.default_rng(17)
    sides = [48, 64, 96, 100, 128, 160, 180, 250, 256, 400, 1000, 1024, 2000, 2048, 3000, 4000, 4096]
    for _ in range(150):
        Nx, Ny = (int(v) for v in rng.choice(sides, 2))
        pad = int(rng.choice([1, 2])) if min(Nx, Ny) >= 64 else 2
        dx = float(rng.uniform(0.2e-6, 4e-6))
        z = float(10 ** rng.uniform(-5, -0.5))
        lam = float(rng.uniform(380e-9, 780e-9))
        g = Geometry.make(Nx, dx, z, [lam], pad=pad, Ny=Ny)
        kx, ky, m = band_limits_xy(g)
        ex, ey = oracle.kmax_rect(pad * Ny, pad * Nx, dx, z, lam)
        assert (int(kx[0]), int(ky[0])) == (ex, ey), (Nx, Ny, pad)
        if Nx != Ny:
            assert int(m[0]) == oracle.mev_rect(pad * Ny, pad * Nx, dx, lam)[2], (Nx, Ny, pad)
        else:
            k1, m1 = band_limits(g)
            assert int(kx[0]) == int(ky[0]) == int(k1[0]) and int(m[0]) == int(m1[0])


@pytest.mark.parametrize(
    "g",
    [_geom(N=49), _geom(N=8), _geom(N=278, pad=1), _geom(N=4106), _geom(N=36000), _geom(N=4192), _geom(N=262, pad=1),
     _geom(dx=0.0), _geom(z=-1.0), _geom(lambdas=[0.0]), _geom(n_index=0.5), _geom(lambdas=np.full(65, 5e-7)),
     _geom(N=180, upsample=8)],
)
def test_invalid_geometry_rejected(lib, g):
    c = g.c()
    assert lib.doe_workspace_bytes(ctypes.byref(c), L.DOE_OP_PSF) == 0
    rc = lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 0, None)
    assert rc in (L.DOE_EINVAL, L.DOE_EUNSUPPORTED)


def test_bad_pad_and_unsupported_size(lib):
    g = _geom()
    c = g.c()
    c.pad = 3
    assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 0, None) == L.DOE_EINVAL
    big = _geom(N=32768).c()  # P = 65536 needs the multi-CTA transform
    rc = lib.doe_psf(ctypes.byref(big), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 0, None)
    assert rc in (L.DOE_OK, L.DOE_ENOWS, L.DOE_EUNSUPPORTED)
    # rectangles run on the mixed-radix passes (each side one CTA per transform up to 8192, split
    # over a cluster above, up to 65536), plain incidence, no upsampling, rectangular band
    for kw in (dict(Ny=128), dict(Ny=8000), dict(Ny=4000, N=4200), dict(Ny=8192, N=200), dict(Ny=42880, N=64320)):
        rect = _geom(**kw).c()
        assert lib.doe_workspace_bytes(ctypes.byref(rect), L.DOE_OP_GRAD) > 0, kw
        assert lib.doe_psf(ctypes.byref(rect), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 0, None) == L.DOE_ENOWS
    for kw in (dict(Ny=70000), dict(Ny=262), dict(Ny=128, upsample=2), dict(Ny=128, bandlimit="circular"),
               dict(Ny=128, theta_x=0.01), dict(Ny=128, src_d=0.1)):
        c = _geom(**kw).c()
        assert lib.doe_workspace_bytes(ctypes.byref(c), L.DOE_OP_PSF) == 0, kw
        assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 0, None) == L.DOE_EUNSUPPORTED, kw


def test_workspace_checked_before_launch(lib):
    g = _geom()
    c = g.c()
    need = lib.doe_workspace_bytes(ctypes.byref(c), L.DOE_OP_PSF)
    assert need > 0
    assert lib.doe_workspace_bytes(ctypes.byref(c), L.DOE_OP_GRAD) > need
    # too small, NULL, misaligned: refused without touching the device
    assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), ctypes.c_void_p(256), need - 1, None) == L.DOE_ENOWS
    assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, need, None) == L.DOE_ENOWS
    assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), ctypes.c_void_p(256 + 8), need, None) == L.DOE_ENOWS


def test_null_pointers_and_bad_mode(lib):
    c = _geom().c()
    assert lib.doe_psf(ctypes.byref(c), None, None, ctypes.c_void_p(16), None, 0, None) == L.DOE_EINVAL
    assert lib.doe_psf(ctypes.byref(c), ctypes.c_void_p(16), None, None, None, 0, None) == L.DOE_EINVAL
    assert lib.doe_grad(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), 7, ctypes.c_void_p(16), None, 1, None, 0, None) == L.DOE_EINVAL
    assert lib.doe_grad(ctypes.byref(c), ctypes.c_void_p(16), None, ctypes.c_void_p(16), 0, ctypes.c_void_p(16), None, 2, None, 0, None) == L.DOE_EINVAL


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert lib.doe_strerror(code)


@pytest.mark.parametrize("N,pad", [(48, 2), (180, 2), (1800, 2), (3600, 1), (4000, 2), (4050, 2), (360, 1),
                                   (4500, 2), (14400, 2), (20000, 2), (13122, 1), (670, 2), (8040, 2)])
def test_mixed_radix_sizes_accepted(lib, N, pad):
    # even N with P = pad N = 2^a 3^b 5^c: one CTA per transform up to 8192, a cluster of Q CTAs
    # above (Table 2's 3600, 28800 and 40000 grids among them)
    c = _geom(N=N, pad=pad).c()
    P = pad * N
    need = lib.doe_workspace_bytes(ctypes.byref(c), L.DOE_OP_PSF)
    assert need >= P * P * 8 + N * P * 8  # natural-layout field buffers, no band compaction
    cg = _geom(N=N, pad=pad, lambdas=[450e-9, 650e-9]).c()
    assert lib.doe_workspace_bytes(ctypes.byref(cg), L.DOE_OP_GRAD) > 2 * need - 2 * N * P * 8


def test_wait_check_rejects_bad_bounds(lib):
    # validated before any launch
    assert lib.doe_check_wait_timeout(0, None) == L.DOE_EINVAL
    assert lib.doe_check_wait_timeout((1 << 20) + 1, None) == L.DOE_EINVAL
