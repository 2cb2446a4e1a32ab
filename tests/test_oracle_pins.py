"""Pins for the FP64 oracle against things other than itself: brute force, closed forms,
invariants, an independent physical model, and the paper's printed grid sizes."""
import os

import numpy as np
import pytest

import oracle
from paper_2505_22313_b300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(7)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 12, 15, 16, 30, 32, 64, 67])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_matches_brute_force_dft(n, inverse):
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # brute force written here: sum_j x_j exp(-+2 pi i j k / n)
    s = 1.0 if inverse else -1.0
    jk = np.outer(np.arange(n), np.arange(n))
    ref = (x[None, :] * np.exp(s * 2j * np.pi * jk / n)).sum(axis=1)
    got = oracle.fft(x, inverse=inverse)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    assert np.abs(oracle.dft(x, inverse=inverse) - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [128, 720, 1024, 3600, 4096, 8040, 5360, 85760, 128640])
def test_fft_matches_numpy(n):
    # 128640 and 85760: Table 2's large-area sides (factor 67), transformed whole by the oracle
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel_l2(oracle.fft(x), np.fft.fft(x)) < 1e-12
    assert rel_l2(oracle.fft(x, inverse=True), np.fft.ifft(x) * n) < 1e-12


def test_fft2_non_square_brute_force():
    ny, nx = 8, 32
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    y = np.arange(ny)
    x = np.arange(nx)
    Wy = np.exp(-2j * np.pi * np.outer(y, y) / ny)
    Wx = np.exp(-2j * np.pi * np.outer(x, x) / nx)
    ref = np.zeros_like(a)
    for l in range(ny):
        for k in range(nx):
            ref[l, k] = (a * Wy[l][:, None] * Wx[k][None, :]).sum()
    assert rel_l2(oracle.fft2(a), ref) < 1e-13


def test_fft_roundtrip_identity():
    n = 2048
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    back = oracle.fft(oracle.fft(x), inverse=True) / n
    assert rel_l2(back, x) < 1e-14


# ------------------------------------------------------------------ band limit
def _local_freq(u, lam, z):
    """Local frequency (cycles per unit u) of the ASM phase 2 pi z sqrt(1/lam^2 - u^2) along u,
    by a centred FP64 difference of the phase -- independent of the closed form f_lim."""
    phase = lambda v: z * np.sqrt(1.0 / lam**2 - v * v)  # phase / (2 pi)
    d = 1e-6 * max(abs(u), 1.0)
    return abs(phase(u + d) - phase(u - d)) / (2 * d)


@pytest.mark.parametrize(
    "N,dx,z,lam",
    [(256, 2e-6, 20e-3, 550e-9), (4096, 1e-6, 50e-3, 450e-9), (4096, 1e-6, 50e-3, 650e-9),
     (8192, 1e-6, 50e-3, 550e-9), (512, 1e-6, 5e-3, 700e-9), (1024, 0.5e-6, 10e-3, 520.6e-9)],
)
def test_kmax_is_the_nyquist_limit_of_the_transfer_phase(N, dx, z, lam):
    P = 2 * N
    du = 1.0 / (P * dx)
    k = oracle.kmax(lam, dx, P, z)
    nyq = 1.0 / (2 * du)
    if k < P // 2:
        # the last kept index is sampled at or under Nyquist, the first dropped one above
        assert _local_freq(k * du, lam, z) <= nyq * (1 + 1e-9)
        assert _local_freq((k + 1) * du, lam, z) > nyq * (1 - 1e-9)
    else:
        assert _local_freq((P // 2) * du, lam, z) <= nyq * (1 + 1e-9)


def test_kmax_config_values():
    # values of the band limit for the stated workloads (C1, C2, C3)
    assert oracle.kmax(550e-9, 2e-6, 512, 20e-3) == 47
    assert [oracle.kmax(l, 1e-6, 8192, 50e-3) for l in (450e-9, 550e-9, 650e-9)] == [1486, 1216, 1028]
    assert [oracle.kmax(l, 1e-6, 16384, 50e-3) for l in (450e-9, 550e-9, 650e-9)] == [5886, 4816, 4075]
    assert oracle.kmax(550e-9, 1e-6, 65536, 100e-3) == 32768  # inactive at the large-area grid


def test_band_mask_integer_rules():
    P, dx, z, lam = 64, 0.25e-6, 5e-6, 700e-9  # fine pitch: the evanescent cut is active
    m = oracle.band_mask(P, dx, z, lam)
    k = oracle.kmax(lam, dx, P, z)
    du = 1.0 / (P * dx)
    kt = np.where(np.arange(P) < P // 2, np.arange(P), np.arange(P) - P)
    prop = (lam**2) * ((kt[None, :] * du) ** 2 + (kt[:, None] * du) ** 2) < 1.0
    inband = (np.abs(kt[None, :]) <= k) & (np.abs(kt[:, None]) <= k)
    assert np.array_equal(m.astype(bool), prop & inband)
    assert (~prop).any()  # the case really exercises the evanescent cut


# ------------------------------------------------------------------ circular band limit
def _flim(lam, du, z):
    return 1.0 / (lam * np.sqrt((2 * du * z) ** 2 + 1))


@pytest.mark.parametrize("P,dx,z,lam", [(64, 0.25e-6, 5e-6, 700e-9), (512, 2e-6, 20e-3, 550e-9),
                                        (256, 1e-6, 2e-3, 450e-9), (96, 1e-6, 1e-3, 633e-9)])
def test_circular_band_mask_rules(P, dx, z, lam):
    # the disc fx^2 + fy^2 < f_lim^2 (and the evanescent cut), written out in floating point
    # here, against the oracle's integer rule m < ceil((f_lim / du)^2); the disc is inside the
    # square band and symmetric under swapping the axes
    m = oracle.band_mask(P, dx, z, lam, bandlimit="circular").astype(bool)
    sq = oracle.band_mask(P, dx, z, lam).astype(bool)
    du = 1.0 / (P * dx)
    kt = np.where(np.arange(P) < P // 2, np.arange(P), np.arange(P) - P).astype(np.float64)
    fx, fy = kt[None, :] * du, kt[:, None] * du
    disc = fx * fx + fy * fy < _flim(lam, du, z) ** 2
    prop = lam**2 * (fx * fx + fy * fy) < 1.0
    assert np.array_equal(m, disc & prop)
    assert np.array_equal(m & sq, m) and (sq & ~m).any()  # strictly inside the square
    assert np.array_equal(m, m.T)
    assert oracle.m_lim(lam, dx, P, z, "circular") <= oracle.m_ev(lam, dx, P)


def test_circular_band_plane_waves_closed_form():
    # pad = 1, flat plate lit by a plane wave on an exact spectral line (kx, ky): inside the disc
    # ASM multiplies it by H(fx, fy); outside the disc but inside the square the circular band
    # removes it entirely, while the square band keeps it
    N, dx, lam, z, c = 64, 1e-6, 550e-9, 200e-6, 0.3e-6
    du = 1.0 / (N * dx)
    r = _flim(lam, du, z) / du  # disc radius in bins (18.4)
    k = oracle.kmax(lam, dx, N, z)
    inside, outside = (int(0.5 * r), -int(0.4 * r)), (k, -k)  # the square's corner lies outside the disc
    assert inside[0] ** 2 + inside[1] ** 2 < r * r < outside[0] ** 2 + outside[1] ** 2
    h = np.full((N, N), c, np.float32)
    for (mx, my), kept in ((inside, True), (outside, False)):
        e_in = oracle.incident(N, dx, lam, np.arcsin(mx * lam / (N * dx)), np.arcsin(my * lam / (N * dx)))
        ph = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z * np.sqrt(1 / lam**2 - (mx * du) ** 2 - (my * du) ** 2)
        ref = np.exp(1j * ph) * e_in
        e_c = oracle.propagate(h, dx, z, lam, n_index=1.46, pad=1, e_in=e_in, bandlimit="circular")
        e_s = oracle.propagate(h, dx, z, lam, n_index=1.46, pad=1, e_in=e_in)
        assert np.abs(e_s - ref).max() < 1e-9
        assert np.abs(e_c - (ref if kept else 0.0)).max() < 1e-9


@pytest.mark.parametrize("N", [128, 90])
def test_parseval_over_circular_band(N):
    dx, z, lam = 1e-6, 5e-3, 550e-9
    P = 2 * N
    h = inputs.heights(N, 12)
    e = oracle.propagate(h, dx, z, lam, bandlimit="circular")
    epad = np.zeros((P, P), np.complex128)
    epad[N // 2:N // 2 + N, N // 2:N // 2 + N] = np.exp(1j * 2 * np.pi * 0.46 * h.astype(np.float64) / lam)
    U = np.fft.fft2(epad)
    du = 1.0 / (P * dx)
    kt = np.fft.fftfreq(P, 1.0 / P)
    disc = (kt[None, :] * du) ** 2 + (kt[:, None] * du) ** 2 < _flim(lam, du, z) ** 2
    lhs = (np.abs(e) ** 2).sum()
    rhs = (np.abs(U[disc]) ** 2).sum() / P**2
    assert abs(lhs - rhs) / rhs < 1e-12
    # the disc keeps less energy than the square band of the same f_lim
    assert lhs < (np.abs(oracle.propagate(h, dx, z, lam)) ** 2).sum()


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("P,z,lam", [(16, 20e-3, 550e-9), (64, 0.1, 550e-9), (256, 50e-3, 450e-9), (1024, 0.1, 650e-9),
                                     (48, 20e-3, 550e-9), (720, 50e-3, 450e-9)])
def test_flat_plate(P, z, lam):
    # h = c everywhere, pad = 1: the spectrum is a DC delta, so E_out = exp(i(k' c + 2 pi z / lam))
    c = 0.37e-6
    h = np.full((P, P), c, np.float32)
    e = oracle.propagate(h, 1e-6, z, lam, n_index=1.46, pad=1)
    phase = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z / lam
    ref = np.exp(1j * np.fmod(phase, 2 * np.pi))
    assert np.abs(e - ref).max() < 1e-8


def test_gaussian_beam_paraxial():
    # E_in = exp(-r^2/w0^2), h = 0; paraxial closed form of a Gaussian beam after z
    N, P, dx, lam, z, w0 = 2048, 4096, 1e-6, 550e-9, 50e-3, 100e-6
    e_in = inputs.gaussian_beam(N, dx, w0)
    e = oracle.propagate(np.zeros((N, N), np.float32), dx, z, lam, pad=2, e_in=e_in)
    k = 2 * np.pi / lam
    zr = np.pi * w0**2 / lam
    w = w0 * np.sqrt(1 + (z / zr) ** 2)
    R = z * (1 + (zr / z) ** 2)
    psi = np.arctan(z / zr)
    c = (np.arange(P) - P // 2) * dx
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    ref = (w0 / w) * np.exp(-r2 / w**2) * np.exp(1j * (np.fmod(k * z, 2 * np.pi) + k * r2 / (2 * R) - psi))
    assert rel_l2(e, ref) < 5e-6  # measured 8.2e-7; non-paraxial terms ~1e-6


# ------------------------------------------------------------------ rectangular grids
@pytest.mark.parametrize("Py,Px,dx,lam", [(96, 160, 1e-6, 550e-9), (64, 48, 0.25e-6, 700e-9), (6000, 8000, 1e-6, 450e-9),
                                          (120, 200, 0.3e-6, 400e-9)])
def test_rect_evanescent_integer_rule(Py, Px, dx, lam):
    # kx^2 B^2 + ky^2 A^2 < ceil((Px Py dx / (g lambda))^2) against lambda^2 (fx^2 + fy^2) < 1
    # in floating point (they agree away from exact ties, and no sample sits on one here)
    a2, b2, mev = oracle.mev_rect(Py, Px, dx, lam)
    g = np.gcd(Px, Py)
    assert a2 == (Px // g) ** 2 and b2 == (Py // g) ** 2
    kx = np.where(np.arange(Px) < Px // 2, np.arange(Px), np.arange(Px) - Px).astype(np.int64)
    ky = np.where(np.arange(Py) < Py // 2, np.arange(Py), np.arange(Py) - Py).astype(np.int64)
    m = kx[None, :] ** 2 * b2 + ky[:, None] ** 2 * a2
    q = lam**2 * ((kx[None, :] / (Px * dx)) ** 2 + (ky[:, None] / (Py * dx)) ** 2)
    assert np.array_equal(m < mev, q < 1.0)
    mask = oracle.band_mask_rect(Py, Px, dx, 1e-9, lam)  # z -> 0: the band limit is inactive
    assert np.array_equal(mask.astype(bool), q < 1.0)



def test_rect_oracle_reduces_to_the_square_one():
    # the rectangular rules (per-axis band, the gcd form of the evanescent cut) and its Python
    # assembly of the chain against the C oracle's square path (its own H and chain)
    for N, pad, dx, z, lam, bl in ((64, 2, 1e-6, 2e-3, 550e-9, True), (90, 2, 0.5e-6, 1e-3, 450e-9, True),
                                   (48, 1, 1e-6, 5e-3, 650e-9, False)):
        h = inputs.heights(N, 30 + N)
        a = oracle.propagate_rect(h, dx, z, lam, pad=pad, bandlimit=bl)
        b = oracle.propagate(h, dx, z, lam, pad=pad, bandlimit=bl)
        assert rel_l2(a, b) < 1e-11  # FP64 rounding of two FFT algorithms (measured <= 1.9e-12)
        assert np.array_equal(oracle.transfer_rect(pad * N, pad * N, dx, z, lam, bl) != 0,
                              oracle.band_mask(pad * N, dx, z, lam, bl).astype(bool))


def test_rect_tilted_flat_plate_closed_form():
    # pad 1, flat plate, a plane wave on exact spectral lines of a 48 x 80 grid: ASM multiplies it
    # by H(mx / (Px dx), my / (Py dx)) with each axis's own step
    Ny, Nx, dx, lam, z, c = 48, 80, 1e-6, 550e-9, 200e-6, 0.3e-6
    for mx, my in ((5, -3), (-12, 7)):
        sx, sy = mx * lam / (Nx * dx), my * lam / (Ny * dx)
        yy = (np.arange(Ny) - Ny // 2)[:, None] * dx
        xx = (np.arange(Nx) - Nx // 2)[None, :] * dx
        e_in = np.exp(2j * np.pi * (xx * sx + yy * sy) / lam)
        e = oracle.propagate_rect(np.full((Ny, Nx), c, np.float32), dx, z, lam, pad=1, e_in=e_in)
        fx, fy = mx / (Nx * dx), my / (Ny * dx)
        ph = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z * np.sqrt(1 / lam**2 - fx**2 - fy**2)
        assert np.abs(e - np.exp(1j * ph) * e_in).max() < 1e-9


def test_rect_band_limit_per_axis_and_parseval():
    Ny, Nx, dx, z, lam = 96, 64, 1e-6, 5e-3, 550e-9
    Py, Px = 2 * Ny, 2 * Nx
    H = oracle.transfer_rect(Py, Px, dx, z, lam)
    kx = np.abs(np.fft.fftfreq(Px, 1.0 / Px))
    ky = np.abs(np.fft.fftfreq(Py, 1.0 / Py))
    # the band's extent along each axis is that axis's square-grid kmax (C oracle)
    assert kx[(H != 0).any(axis=0)].max() == oracle.kmax(lam, dx, Px, z)
    assert ky[(H != 0).any(axis=1)].max() == oracle.kmax(lam, dx, Py, z)
    h = inputs.heights(96, 33)[:, :64]
    e = oracle.propagate_rect(h, dx, z, lam)
    Ep = np.zeros((Py, Px), np.complex128)
    Ep[Ny // 2:Ny // 2 + Ny, Nx // 2:Nx // 2 + Nx] = np.exp(1j * 2 * np.pi * 0.46 * h.astype(np.float64) / lam)
    U = np.fft.fft2(Ep)
    lhs = (np.abs(e) ** 2).sum()
    rhs = (np.abs(U[H != 0]) ** 2).sum() / (Px * Py)
    assert abs(lhs - rhs) / rhs < 1e-12 and lhs <= Nx * Ny * (1 + 1e-12)


def test_rect_gradient_matches_central_differences():
    Ny, Nx, dx, z = 6, 4, 2e-6, 1e-3
    lams = [450e-9, 650e-9]
    h = inputs.heights(8, 34)[:Ny, :Nx]
    T = rng.random((2, 2 * Ny, 2 * Nx)) * 0.5
    g, loss = oracle.grad_rect(h, dx, z, lams, T)
    h64 = h.astype(np.float64)

    def lossf(hh):  # FP64 heights are used as they are
        return sum(float(((np.abs(oracle.propagate_rect(hh, dx, z, lam)) ** 2 - T[j]) ** 2).sum())
                   for j, lam in enumerate(lams))

    eps = 1e-11
    fd = np.zeros((Ny, Nx))
    for i in range(Ny):
        for j in range(Nx):
            hp = h64.copy(); hp[i, j] += eps
            hm = h64.copy(); hm[i, j] -= eps
            fd[i, j] = (lossf(hp) - lossf(hm)) / (2 * eps)
    assert abs(lossf(h64) - loss) <= 1e-12 * loss
    assert rel_l2(g, fd) < 1e-5


# ------------------------------------------------------------------ incident fields
def test_incident_tilt_is_one_spectral_line():
    # sin(theta) = m lambda / (N dx) puts the tilted plane wave on DFT bin m of each axis, with
    # value N^2 (-1)^(mx + my) (phase referenced to sample N/2); numpy's FFT, not the oracle's
    N, dx, lam = 64, 1e-6, 550e-9
    for mx, my in ((5, 0), (0, -3), (7, -2)):
        e = oracle.incident(N, dx, lam, np.arcsin(mx * lam / (N * dx)), np.arcsin(my * lam / (N * dx)))
        F = np.fft.fft2(e)
        ref = np.zeros((N, N), np.complex128)
        ref[my % N, mx % N] = N * N * (-1.0) ** (mx + my)
        assert np.abs(F - ref).max() < 1e-9 * N * N


def test_incident_tilted_flat_plate_closed_form():
    # pad = 1, flat plate, a plane wave on an exact spectral line: ASM multiplies it by
    # H(fx, fy) = exp(i 2 pi z sqrt(1 / lambda^2 - fx^2 - fy^2)) and nothing else
    N, dx, lam, z, c = 64, 1e-6, 550e-9, 200e-6, 0.3e-6
    du = 1.0 / (N * dx)
    for mx, my in ((5, -3), (-12, 9)):
        e_in = oracle.incident(N, dx, lam, np.arcsin(mx * lam / (N * dx)), np.arcsin(my * lam / (N * dx)))
        e = oracle.propagate(np.full((N, N), c, np.float32), dx, z, lam, n_index=1.46, pad=1, e_in=e_in)
        ph = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z * np.sqrt(1 / lam**2 - (mx * du) ** 2 - (my * du) ** 2)
        assert np.abs(e - np.exp(1j * ph) * e_in).max() < 1e-9


def test_incident_spherical_paraxial_limit_and_conjugate():
    # near the axis the spherical wave is the Fresnel quadratic phase with amplitude ~ 1:
    # |phase - pi rho^2 / (lambda d)| <= k rho^4 / (8 d^3), |amp - 1 + rho^2 / (2 d^2)| <= 3 rho^4 / (8 d^4)
    N, dx, lam, d = 64, 1e-6, 550e-9, 10e-3
    e = oracle.incident(N, dx, lam, d=d)
    c = (np.arange(N) - N // 2) * dx
    rho2 = c[:, None] ** 2 + c[None, :] ** 2
    k = 2 * np.pi / lam
    dph = np.angle(e * np.exp(-1j * np.pi * rho2 / (lam * d)))
    # (+1e-10: FP64 rounding of r - |d| is k ulp(d) ~ 2e-11 rad)
    assert np.all(np.abs(dph) <= k * rho2**2 / (8 * d**3) * 1.001 + 1e-10)
    assert np.abs(dph).max() > 1e-6  # the quartic term is visible: the wave is not the paraxial one
    assert np.all(np.abs(np.abs(e) - 1 + rho2 / (2 * d * d)) <= 3 * rho2**2 / (8 * d**4) + 1e-15)
    # a converging wave is the conjugate of the diverging one
    assert np.array_equal(oracle.incident(N, dx, lam, d=-d), np.conj(e))


def test_converging_wave_focuses_where_geometry_says():
    # flat DOE lit by a wave converging to distance z: the PSF at z peaks on the optical axis
    # (padded index P/2); a tilt of the same wave moves the focus to z tan(theta) on its axis
    N, dx, lam, z = 256, 1e-6, 550e-9, 2e-3
    P = 2 * N
    h = np.zeros((N, N), np.float32)
    I0 = oracle.psf(h, dx, z, [lam], e_in=oracle.incident(N, dx, lam, d=-z))[0]
    assert np.unravel_index(I0.argmax(), I0.shape) == (P // 2, P // 2)
    Id = oracle.psf(h, dx, z, [lam], e_in=oracle.incident(N, dx, lam, d=z))[0]
    assert I0.max() > 20 * Id.max()  # the diverging wave does not focus
    tx, ty = 0.02, -0.015
    It = oracle.psf(h, dx, z, [lam], e_in=oracle.incident(N, dx, lam, np.arcsin(tx), np.arcsin(ty), d=-z))[0]
    py, px = np.unravel_index(It.argmax(), It.shape)
    ex = z * tx / np.sqrt(1 - tx * tx) / dx
    ey = z * ty / np.sqrt(1 - ty * ty) / dx
    assert abs(px - P // 2 - ex) <= 1.0 and abs(py - P // 2 - ey) <= 1.0


@pytest.mark.parametrize("N", [128, 180])
def test_parseval_over_band(N):
    dx, z, lam = 1e-6, 5e-3, 550e-9
    P = 2 * N
    h = inputs.heights(N, 11)
    e = oracle.propagate(h, dx, z, lam)
    # independent route: numpy FFT of the padded field, band from the stated integer rules
    epad = np.zeros((P, P), np.complex128)
    epad[N // 2:N // 2 + N, N // 2:N // 2 + N] = np.exp(1j * 2 * np.pi * 0.46 * h.astype(np.float64) / lam)
    U = np.fft.fft2(epad)
    du = 1.0 / (P * dx)
    kt = np.fft.fftfreq(P, 1.0 / P)
    flim = 1.0 / (lam * np.sqrt((2 * du * z) ** 2 + 1))
    inband = (np.abs(kt)[None, :] * du < flim) & (np.abs(kt)[:, None] * du < flim)
    lhs = (np.abs(e) ** 2).sum()
    rhs = (np.abs(U[inband]) ** 2).sum() / P**2
    assert abs(lhs - rhs) / rhs < 1e-12
    assert lhs <= N * N * (1 + 1e-12)


@pytest.mark.parametrize("N,w2", [(32, 36.0), (24, 20.0)])
def test_rayleigh_sommerfeld_direct_sum(N, w2):
    # smooth apodised field whose spectrum lies inside the band: ASM ~ RS-I direct sum
    # (N = 24: a 48 x 48 grid, mixed-radix transforms)
    P, dx, lam, z = 2 * N, 0.5e-6, 550e-9, 50e-6
    yy, xx = np.mgrid[0:N, 0:N]
    r2 = (yy - N / 2) ** 2 + (xx - N / 2) ** 2
    amp = np.exp(-r2 / w2)
    h = (0.3e-6 * np.exp(-r2 / 200.0)).astype(np.float32)
    e_doe = amp * np.exp(1j * 2 * np.pi * 0.46 * h.astype(np.float64) / lam)
    e_asm = oracle.propagate(h, dx, z, lam, pad=2, e_in=amp)
    e_rs = oracle.rs_direct(e_doe, P, dx, z, lam)
    err = rel_l2(e_asm, e_rs)
    assert err < 1e-3, err  # measured 2.1e-4
    # a flipped sign convention or a missing transfer function fails by orders of magnitude
    e_conj = oracle.propagate(h, dx, -z, lam, pad=2, e_in=amp)
    assert rel_l2(e_conj, e_rs) > 0.1


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("N", [8, 6])
def test_gradient_matches_fp64_central_differences(N):
    dx, z = 2e-6, 1e-3
    lams = np.array([450e-9, 650e-9])
    P = 2 * N
    h = inputs.heights(N, 21)
    T = rng.random((2, P, P)).astype(np.float32) * 0.5
    g, loss = oracle.grad(h, dx, z, lams, T)
    h64 = h.astype(np.float64)
    assert abs(oracle.loss_l2(h64, dx, z, lams, T) - loss) <= 1e-12 * loss
    eps = 1e-11
    fd = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            hp = h64.copy(); hp[i, j] += eps
            hm = h64.copy(); hm[i, j] -= eps
            fd[i, j] = (oracle.loss_l2(hp, dx, z, lams, T) - oracle.loss_l2(hm, dx, z, lams, T)) / (2 * eps)
    assert rel_l2(g, fd) < 1e-5


def test_gradient_vjp_mode_equals_l2_mode():
    N, dx, z, lam = 16, 1e-6, 2e-3, 550e-9
    P = 2 * N
    h = inputs.heights(N, 22)
    T = rng.random((1, P, P)).astype(np.float32)
    g_l2, _ = oracle.grad(h, dx, z, [lam], T)
    I = oracle.psf(h, dx, z, [lam])
    G = (2.0 * (I - T.astype(np.float64))).astype(np.float32)
    g_vjp, _ = oracle.grad(h, dx, z, [lam], G, mode="vjp")
    assert rel_l2(g_vjp, g_l2) < 1e-6  # G is rounded to float32


def test_exact_difference_fd_matches_plain_fd():
    N, dx, z = 16, 1e-6, 2e-3
    lams = np.array([500e-9])
    P = 2 * N
    h = inputs.heights(N, 23)
    T = rng.random((1, P, P)).astype(np.float32)
    py = np.array([0, 3, 7, 15]); px = np.array([5, 8, 0, 15])
    eps = 1e-10
    fd = oracle.fd_exact(h, dx, z, lams, T, py, px, eps)
    h64 = h.astype(np.float64)
    for q in range(py.size):
        hp = h64.copy(); hp[py[q], px[q]] += eps
        hm = h64.copy(); hm[py[q], px[q]] -= eps
        ref = (oracle.loss_l2(hp, dx, z, lams, T) - oracle.loss_l2(hm, dx, z, lams, T)) / (2 * eps)
        assert abs(fd[q] - ref) <= 1e-6 * abs(ref) + 1e-9


# ------------------------------------------------------------------ render / Wiener
def test_render_matches_direct_sum():
    C, H, W, Pp = 2, 8, 16, 32
    psf = rng.random((C, Pp, Pp)).astype(np.float32)
    img = rng.random((C, H, W)).astype(np.float32)
    out = oracle.render(psf, img)
    for c in range(C):
        k = psf[c, Pp // 2 - H // 2:Pp // 2 - H // 2 + H, Pp // 2 - W // 2:Pp // 2 - W // 2 + W].astype(np.float64)
        k = k / k.sum()
        ref = np.zeros((H, W))
        for y in range(H):
            for x in range(W):
                s = 0.0
                for u in range(H):
                    for v in range(W):
                        yy, xx = y + H // 2 - u, x + W // 2 - v
                        if 0 <= yy < H and 0 <= xx < W:
                            s += img[c, yy, xx] * k[u, v]
                ref[y, x] = s
        assert rel_l2(out[c], ref) < 1e-13


def test_wiener_inverts_a_circular_blur():
    C, H, W, Pp = 1, 16, 16, 32
    k = np.zeros((Pp, Pp), np.float32)
    k[Pp // 2, Pp // 2] = 4.0
    k[Pp // 2 + 1, Pp // 2] = 1.0
    k[Pp // 2, Pp // 2 - 1] = 0.5
    psf = k[None]
    x = rng.random((C, H, W))
    kc = psf[0, Pp // 2 - H // 2:Pp // 2 + H // 2, Pp // 2 - W // 2:Pp // 2 + W // 2].astype(np.float64)
    kc /= kc.sum()
    y = np.zeros((C, H, W))
    for yy in range(H):  # circular blur by brute force, kernel centre at (H/2, W/2)
        for xx in range(W):
            for u in range(H):
                for v in range(W):
                    y[0, yy, xx] += kc[u, v] * x[0, (yy - (u - H // 2)) % H, (xx - (v - W // 2)) % W]
    xh = oracle.wiener(psf, y.astype(np.float32), 1e-12)
    assert rel_l2(xh, x) < 1e-5  # limited by the float32 rounding of y


# ------------------------------------------------------------------ consistency + paper grids
def test_psf_rows_equal_full_psf():
    N, dx, z, lam = 32, 1e-6, 3e-3, 600e-9
    h = inputs.heights(N, 24)
    full = oracle.psf(h, dx, z, [lam])[0]
    rows = np.array([0, 5, 31, 32, 63])
    part = oracle.psf_rows(h, dx, z, lam, rows)
    assert np.abs(part - full[rows]).max() <= 1e-12 * full.max()


@pytest.mark.parametrize("z,with_ein", [(3e-3, False), (2e-4, True)])
def test_grad_rows_equal_masked_full_gradient(z, with_ein):
    # the row-subset adjoint (used where the FP64 field does not fit host memory) equals the
    # full-grid gradient, itself pinned to central differences above, when dL/dI vanishes
    # off the chosen output rows; first case has an active band limit (kmax = 1)
    N, dx, lam = 32, 1e-6, 600e-9
    P = 2 * N
    h = inputs.heights(N, 25)
    r = np.random.default_rng(26)
    e_in = (r.random((N, N)) + 1j * r.random((N, N))) if with_ein else None
    rows = np.array([0, 5, 31, 32, 40, 63])
    G = np.zeros((1, P, P), np.float32)
    G[0, rows] = r.standard_normal((rows.size, P)).astype(np.float32)
    full, _ = oracle.grad(h, dx, z, [lam], G, mode="vjp", e_in=e_in)
    drows = np.array([0, 3, 16, 31])
    part = oracle.grad_rows(h, dx, z, lam, rows, G[0, rows], drows, e_in=e_in)
    assert np.abs(part - full[drows]).max() <= 1e-12 * np.abs(full).max()


def test_upsample_nearest_and_its_adjoint():
    # brute force on a small layout, and <up(a), b> = <a, up^T(b)> (dot-product test)
    r = np.random.default_rng(40)
    for f in (1, 2, 4, 8):
        a = r.random((3, 3)).astype(np.float32)
        up = oracle.upsample_nearest(a, f)
        assert up.shape == (3 * f, 3 * f)
        for i in range(3 * f):
            for x in range(3 * f):
                assert up[i, x] == a[i // f, x // f]
        b = r.standard_normal((3 * f, 3 * f))
        lhs = float((up.astype(np.float64) * b).sum())
        rhs = float((a.astype(np.float64) * oracle.layout_grad(b, f)).sum())
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-12
        bs = oracle.layout_grad(b, f)
        for ic in range(3):
            for xc in range(3):
                assert abs(bs[ic, xc] - b[ic * f:(ic + 1) * f, xc * f:(xc + 1) * f].sum()) < 1e-12


def test_adam_first_step_scale_invariance_and_descent():
    r = np.random.default_rng(41)
    g = r.standard_normal(64)
    z = np.zeros(64)
    lr, eps = 1e-3, 1e-12
    # first step from zero moments: the bias-corrected step is lr g / (|g| + eps) = lr sign(g)
    free = dict(h_min=-np.inf, h_max=np.inf)  # no projection for these checks
    h1, _, _ = oracle.adam_step(z, g, z, z, lr, 1, eps=eps, **free)
    assert np.allclose(h1, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    # scaling every gradient by c > 0 leaves the steps unchanged (eps negligible)
    ha, ma, va = z, z, z
    hb, mb, vb = z, z, z
    for t in range(1, 6):
        gt = r.standard_normal(64)
        ha, ma, va = oracle.adam_step(ha, gt, ma, va, lr, t, eps=eps, **free)
        hb, mb, vb = oracle.adam_step(hb, 1e3 * gt, mb, vb, lr, t, eps=eps, **free)
    # (the eps term moves each step by at most ~lr eps / sqrt(v_hat) ~ 1e-15 here)
    assert np.abs(ha - hb).max() <= 1e-12
    # on f(x) = x^2 / 2 from x = 1 the iterates decrease towards the minimiser
    x, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 201):
        x_new, m, v = oracle.adam_step(x, x, m, v, 1e-2, t, **free)
        assert x_new[0] < x[0] or x[0] < 2e-2
        x = x_new
    assert abs(x[0]) < 2e-2
    # projection onto the fabricable range
    hc, _, _ = oracle.adam_step(np.array([0.0, 1.0]), np.array([1.0, -1.0]), np.zeros(2), np.zeros(2), 0.5, 1,
                                h_min=0.0, h_max=1.2)
    assert hc[0] == 0.0 and abs(hc[1] - 1.2) < 1e-12


@pytest.mark.parametrize("iters", [3000, 7, 2])
def test_cosine_schedule_pins(iters):
    # Sec. 3.2: the learning rate starts at lr0 and decays to zero over `iters` iterations along
    # a half cosine.  Steps are numbered t = 1 .. iters, so step 1 uses lr0, the midpoint
    # t = iters / 2 + 1 uses lr0 / 2, and the step after the last one would use exactly 0; the
    # last step itself uses lr0 sin^2(pi / (2 iters)) (half-angle identity).
    lr0 = 1e-2
    assert oracle.cosine_lr(lr0, 1, iters) == lr0
    if iters % 2 == 0:
        assert abs(oracle.cosine_lr(lr0, iters // 2 + 1, iters) - 0.5 * lr0) <= 1e-15
    assert abs(oracle.cosine_lr(lr0, iters + 1, iters)) <= 1e-18
    assert abs(oracle.cosine_lr(lr0, iters, iters) - lr0 * np.sin(np.pi / (2 * iters)) ** 2) <= 1e-15
    lrs = [oracle.cosine_lr(lr0, t, iters) for t in range(1, iters + 2)]
    assert all(a > b for a, b in zip(lrs, lrs[1:]))  # strictly decreasing to zero
    # symmetric about the midpoint: lr(t) + lr(iters + 2 - t) = lr0
    assert max(abs(lrs[k] + lrs[iters - k] - lr0) for k in range(iters + 1)) <= 1e-15


def test_lanczos3_upsampling_properties():
    r = np.random.default_rng(42)
    # f = 1 is the identity (the kernel vanishes at non-zero integers and is 1 at 0)
    a = r.random((8, 8))
    assert np.abs(oracle.upsample_lanczos3(a, 1) - a.astype(np.float32)).max() == 0.0
    for f in (2, 4, 8):
        n = 64
        # a constant layout stays constant (normalised weights, clamped edges)
        assert np.abs(oracle.upsample_lanczos3(np.full((n, n), 0.7), f) - np.float32(0.7)).max() < 1e-6
        # a slowly varying layout (periods of 32 and 40 cells) is interpolated at the
        # cell-centre positions to within Lanczos-3's own error there (3.6e-3 at most);
        # sampling it half a fine sample off, or with another kernel, misses by 1.6e-2 or more
        c = np.arange(n)
        lay = np.cos(2 * np.pi * c / 32.0)[:, None] * np.cos(2 * np.pi * c / 40.0)[None, :]
        up = oracle.upsample_lanczos3(lay, f)
        u = (np.arange(n * f) + 0.5) / f - 0.5
        exact = np.cos(2 * np.pi * u / 32.0)[:, None] * np.cos(2 * np.pi * u / 40.0)[None, :]
        inner = slice(4 * f, (n - 4) * f)
        assert np.abs(up[inner, inner] - exact[inner, inner]).max() < 5e-3
        # the layout gradient is the transpose: <up(a), b> = <a, up^T(b)>
        a = r.standard_normal((n, n))
        b = r.standard_normal((n * f, n * f))
        lhs = float((oracle.upsample_lanczos3(a, f).astype(np.float64) * b).sum())
        rhs = float((a * oracle.layout_grad_lanczos3(b, f)).sum())
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)  # the forward output is rounded to float32


def test_radial_parameterisation():
    N = 64
    r = np.random.default_rng(44)
    c = r.standard_normal(9) * 1e-7
    h = oracle.radial_heights(c, N)
    # the axis sample is the piston, the edge midpoints (rho = R) sum the coefficients and the
    # corner (rho^2 = 2 R^2) weighs them by 2^k
    assert h[N // 2, N // 2] == c[0]
    for y, x in ((N // 2, 0), (0, N // 2)):
        assert abs(h[y, x] - c.sum()) <= 1e-22
    assert abs(h[0, 0] - (c * 2.0 ** np.arange(9)).sum()) <= 1e-20
    # symmetric under the 90-degree rotation and the reflections about the axis sample
    a = h[1:, 1:]  # the samples symmetric about (N/2, N/2)
    assert np.array_equal(a, np.rot90(a)) and np.array_equal(a, a[::-1, :]) and np.array_equal(a, a.T)
    # s^1 along the centre row is ((x - N/2) / (N/2))^2
    e1 = oracle.radial_heights([0.0, 1.0], N)
    assert np.allclose(e1[N // 2], ((np.arange(N) - N / 2) / (N / 2)) ** 2, rtol=0, atol=1e-15)
    # the gradient is the transpose: <heights(c), g> = <c, grad(g)>
    g = r.standard_normal((N, N))
    assert abs((h * g).sum() - (c * oracle.radial_grad(g, 9)).sum()) <= 1e-12 * np.abs(h * g).sum()


def test_table2_grids_are_twice_the_design_sample_count():
    rows = np.loadtxt(os.path.join(GOLD, "table2_grids.txt"))
    for ay, ax, pitch, gy, gx in rows:
        ny = round(ay * 1e3 / pitch)
        nx = round(ax * 1e3 / pitch)
        assert (2 * ny, 2 * nx) == (int(gy), int(gx))
