"""Rectangular grids (Nx != Ny) on the CUDA path against the oracle's rectangular
restatement (its own FFT, per-axis band limits and the integer evanescent rule of Sec. 3.1
read for Py != Px): band masks bit-exact, fields, PSFs and gradients element by element,
power-of-two, mixed-radix and mixed power-of-two / mixed-radix sides, both paddings."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_22313_b300 import api, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu

TOL_PSF = 1e-5   # relative L2, PSFs and fields (FP32 path vs FP64 oracle)
TOL_GRAD = 1e-4  # relative L2, gradients


def rel_l2(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2505_22313_b300 import build

    build.build()
    assert torch.cuda.is_available()
    api.init()


def _h(Ny, Nx, seed):
    return np.ascontiguousarray(inputs.heights(max(Nx, Ny), seed)[:Ny, :Nx])


def _target(Py, Px, Ny, Nx, L, seed):
    """Spot-array target of the larger square grid, centre-cropped to Py x Px."""
    P, N = max(Px, Py), max(Nx, Ny)
    T = inputs.spot_target(P, N, L, seed)
    y0, x0 = (P - Py) // 2, (P - Px) // 2
    return np.ascontiguousarray(T[:, y0:y0 + Py, x0:x0 + Px])


# (Ny, Nx, pad): power-of-two sides, mixed-radix sides, one of each; pad 1 and 2
SHAPES = [(64, 128, 2), (96, 160, 2), (160, 96, 2), (180, 128, 2), (200, 360, 1), (256, 48, 2), (90, 250, 2)]


@pytest.mark.parametrize("Ny,Nx,pad", SHAPES)
def test_rect_band_mask_bit_exact(Ny, Nx, pad):
    dx, z = 1e-6, 2e-3
    for lam in (450e-9, 650e-9):
        g = Geometry.make(Nx, dx, z, [lam], pad=pad, Ny=Ny)
        m = api.debug_band_mask(g, 0).cpu().numpy()
        ref = oracle.band_mask_rect(pad * Ny, pad * Nx, dx, z, lam)
        assert m.shape == ref.shape
        assert np.array_equal(m, ref), (Ny, Nx, pad, lam, int((m != ref).sum()))


@pytest.mark.parametrize("Ny,Nx,pad", SHAPES)
def test_rect_propagate_vs_oracle(Ny, Nx, pad):
    dx, z, lams = 1e-6, 2e-3, [450e-9, 633e-9]
    h = _h(Ny, Nx, 12000 + Nx + Ny)
    g = Geometry.make(Nx, dx, z, lams, pad=pad, Ny=Ny)
    E = api.propagate(torch.from_numpy(h).cuda(), g).cpu().numpy()
    assert E.shape == (2, pad * Ny, pad * Nx)
    for j, lam in enumerate(lams):
        ref = oracle.propagate_rect(h, dx, z, lam, pad=pad)
        assert rel_l2(E[j], ref) < TOL_PSF, (j, rel_l2(E[j], ref))


@pytest.mark.parametrize("Ny,Nx,pad", [(96, 160, 2), (180, 128, 2), (200, 360, 1)])
def test_rect_psf_and_grad_vs_oracle(Ny, Nx, pad):
    dx, z = 0.5e-6, 2e-3
    lams = [450e-9, 550e-9, 650e-9]
    Py, Px = pad * Ny, pad * Nx
    h = _h(Ny, Nx, 12100 + Nx)
    T = _target(Py, Px, Ny, Nx, 3, 12200 + Nx)
    g = Geometry.make(Nx, dx, z, lams, pad=pad, Ny=Ny)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    assert I.shape == (3, Py, Px)
    assert rel_l2(I, oracle.psf_rect(h, dx, z, lams, pad=pad)) < TOL_PSF
    gref, lref = oracle.grad_rect(h, dx, z, lams, T, pad=pad)
    for recompute in (True, False):
        ws = None
        if not recompute:  # the fields a PSF call left in a gradient-sized workspace
            ws = api.workspace(api.workspace_bytes(g, 3))
            api.psf(ht, g, ws=ws)
        gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda(), recompute=recompute, ws=ws)
        assert gr.shape == (Ny, Nx)
        err = rel_l2(gr.cpu().numpy(), gref)
        assert err < TOL_GRAD, err
        assert abs(loss.item() - lref) <= 1e-5 * lref


def test_rect_incident_field_and_no_band_limit():
    Ny, Nx, dx, z, lam = 96, 160, 1e-6, 2e-3, 532e-9
    h = _h(Ny, Nx, 12300)
    rng = np.random.default_rng(12301)
    e_in = (rng.standard_normal((Ny, Nx)) + 1j * rng.standard_normal((Ny, Nx))).astype(np.complex64)
    for bl in (True, False):
        g = Geometry.make(Nx, dx, z, [lam], Ny=Ny, bandlimit=bl)
        I = api.psf(torch.from_numpy(h).cuda(), g, e_in=torch.from_numpy(e_in).cuda()).cpu().numpy()
        ref = oracle.psf_rect(h, dx, z, [lam], e_in=e_in.astype(np.complex128), bandlimit=bl)
        assert rel_l2(I, ref) < TOL_PSF, (bl, rel_l2(I, ref))


def test_rect_batched_requests_equal_single_calls():
    Ny, Nx, dx = 96, 160, 1e-6
    hs = [torch.from_numpy(_h(Ny, Nx, 12500 + k)).cuda() for k in range(3)]
    gs = [Geometry.make(Nx, dx, 2e-3, [500e-9], Ny=Ny), Geometry.make(Nx, dx, 3e-3, [600e-9, 700e-9], Ny=Ny),
          Geometry.make(Nx, dx, 2e-3, [450e-9], Ny=Ny)]
    for h, gg, m in zip(hs, gs, api.psf_many(hs, gs)):
        assert torch.equal(m, api.psf(h, gg))


@pytest.mark.parametrize("Ny,Nx", [(3000, 4000), (1024, 4096)])
def test_rect_large_psf_vs_oracle(Ny, Nx):
    """Padded 6000 x 8000 (mixed radix on both axes) and 2048 x 8192 (power-of-two sides at the
    one-CTA limit): full PSFs against the oracle."""
    dx, z, lam = 1e-6, 20e-3, 550e-9
    h = _h(Ny, Nx, 12600 + Ny)
    g = Geometry.make(Nx, dx, z, [lam], Ny=Ny)
    I = api.psf(torch.from_numpy(h).cuda(), g).cpu().numpy()
    ref = oracle.psf_rect(h, dx, z, [lam])
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)


def test_rect_medium_grad_vs_oracle():
    Ny, Nx, dx, z, lams = 1000, 1500, 1e-6, 10e-3, [520.6e-9]
    h = _h(Ny, Nx, 12700)
    T = _target(2 * Ny, 2 * Nx, Ny, Nx, 1, 12701)
    g = Geometry.make(Nx, dx, z, lams, Ny=Ny)
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad_rect(h, dx, z, lams, T)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref


# sides above one CTA's transform: split over a cluster per axis.  (Ny, Nx): the row transform
# split (Px = 9000 = 8 x 1125, 18000 = 8 x 2250 with composite stages), the column transform
# split (Py = 9000, 18000: two columns per cluster), and both.
SPLIT_SHAPES = [(1000, 4500), (4500, 1000), (300, 9000), (9000, 300), (4800, 4500)]


@pytest.mark.parametrize("Ny,Nx", SPLIT_SHAPES)
def test_rect_split_sides_psf_vs_oracle(Ny, Nx):
    dx, z, lam = 1e-6, 10e-3, 550e-9
    h = _h(Ny, Nx, 12800 + Nx + Ny)
    g = Geometry.make(Nx, dx, z, [lam], Ny=Ny)
    I = api.psf(torch.from_numpy(h).cuda(), g).cpu().numpy()
    ref = oracle.psf_rect(h, dx, z, [lam])
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    m = api.debug_band_mask(g, 0).cpu().numpy()
    assert np.array_equal(m, oracle.band_mask_rect(2 * Ny, 2 * Nx, dx, z, lam))


@pytest.mark.parametrize("Ny,Nx", [(500, 4500), (4500, 500)])
def test_rect_split_sides_grad_vs_oracle(Ny, Nx):
    dx, z, lams = 1e-6, 5e-3, [500e-9, 620e-9]
    h = _h(Ny, Nx, 12900 + Nx)
    T = _target(2 * Ny, 2 * Nx, Ny, Nx, 2, 12901 + Nx)
    g = Geometry.make(Nx, dx, z, lams, Ny=Ny)
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad_rect(h, dx, z, lams, T)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref


def _h_uniform(Ny, Nx, seed):
    """Uniform random heights in [0, 1.2 um) for long thin grids (the smoothed square generator
    would build a max(Nx, Ny)^2 map)."""
    return (np.random.default_rng(seed).random((Ny, Nx), dtype=np.float32) * np.float32(1.2e-6)).astype(np.float32)


# Table 2's large-area sides, 128640 = 16 x 8040 and 85760 = 16 x 5360 (prime 67 in both
# sub-transforms, 16-CTA clusters), each against a short other side so that the oracle runs
# in full
@pytest.mark.parametrize("Ny,Nx", [(100, 64320), (42880, 100)])
def test_rect_table2_sides_psf_vs_oracle(Ny, Nx):
    dx, z, lam = 1e-6, 20e-3, 550e-9
    h = _h_uniform(Ny, Nx, 13000 + Ny)
    g = Geometry.make(Nx, dx, z, [lam], Ny=Ny)
    I = api.psf(torch.from_numpy(h).cuda(), g).cpu().numpy()
    ref = oracle.psf_rect(h, dx, z, [lam])
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    m = api.debug_band_mask(g, 0).cpu().numpy()
    assert np.array_equal(m, oracle.band_mask_rect(2 * Ny, 2 * Nx, dx, z, lam))
