"""GPU parity of libdoe against the FP64 oracle (element by element on seeded inputs), plus
closed-form and property checks at sizes the oracle cannot finish quickly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_22313_b300 import api, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu

TOL_PSF = 1e-5   # relative L2, PSFs, fields and renders (FP32 path vs FP64 oracle)
TOL_GRAD = 1e-4  # relative L2, gradients


def rel_l2(a, b):
    a = np.asarray(a, np.float64) if not np.iscomplexobj(a) else np.asarray(a, np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2505_22313_b300 import build

    build.build()
    assert torch.cuda.is_available()
    api.init()


def _h(N, seed):
    return inputs.heights(N, seed)


# -------------------------------------------------------------- fields, every transform size
@pytest.mark.parametrize("N,pad", [(32, 1), (16, 2), (32, 2), (64, 2), (128, 1), (128, 2), (256, 2),
                                   (512, 2), (1024, 2), (2048, 1)])
def test_propagate_matches_oracle_all_sizes(N, pad):
    dx, z = 1e-6, 3e-3 * N / 256
    lams = [450e-9, 633e-9]
    h = _h(N, 1000 + N)
    g = Geometry.make(N, dx, z, lams, pad=pad)
    e = api.propagate(torch.from_numpy(h).cuda(), g).cpu().numpy()
    for j, lam in enumerate(lams):
        ref = oracle.propagate(h, dx, z, lam, pad=pad)
        assert rel_l2(e[j], ref) < TOL_PSF, (N, pad, j, rel_l2(e[j], ref))


def test_psf_config_small_full():
    # 256 x 256 DOE, 2 um pitch, 550 nm, z = 20 mm, 2x padding -> 512 x 512 PSF
    N, dx, z, lam = 256, 2e-6, 20e-3, 550e-9
    h = _h(N, 1001)
    g = Geometry.make(N, dx, z, [lam])
    I = api.psf(torch.from_numpy(h).cuda(), g).cpu().numpy()
    ref = oracle.psf(h, dx, z, [lam])
    err = rel_l2(I, ref)
    assert err < TOL_PSF, err


def test_psf_with_incident_field():
    N, dx, z, lam = 128, 1e-6, 2e-3, 532e-9
    h = _h(N, 77)
    rng = np.random.default_rng(5)
    e_in = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    g = Geometry.make(N, dx, z, [lam])
    I = api.psf(torch.from_numpy(h).cuda(), g, e_in=torch.from_numpy(e_in).cuda()).cpu().numpy()
    ref = oracle.psf(h, dx, z, [lam], e_in=e_in.astype(np.complex128))
    assert rel_l2(I, ref) < TOL_PSF


@pytest.mark.parametrize("N", [512, 2048, 4096, 8192])
def test_flat_plate_closed_form_every_size(N):
    # h = c, pad = 1: E_out = exp(i (k' c + 2 pi z / lambda)) everywhere, I = 1
    c, dx, z, lam = 0.37e-6, 1e-6, 0.1, 550e-9
    h = torch.full((N, N), c, dtype=torch.float32, device="cuda")
    g = Geometry.make(N, dx, z, [lam], pad=1)
    e = api.propagate(h, g)[0]
    phase = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z / lam
    ref = complex(np.cos(np.fmod(phase, 2 * np.pi)), np.sin(np.fmod(phase, 2 * np.pi)))
    err = (e - torch.tensor(ref, dtype=torch.complex64, device="cuda")).abs().max().item()
    assert err < 2e-5, err


@pytest.mark.parametrize("N,lams", [(4096, [450e-9, 550e-9, 650e-9]), (8192, [450e-9, 550e-9, 650e-9])])
def test_psf_large_rows_vs_oracle(N, lams):
    # full-size workloads: exact FP64 rows (seeded subset) from the oracle's row-subset mode
    dx, z = 1e-6, 50e-3
    P = 2 * N
    h = _h(N, 1002 if N == 4096 else 1003)
    g = Geometry.make(N, dx, z, lams)
    I = api.psf(torch.from_numpy(h).cuda(), g)
    rows = np.unique(np.concatenate([np.arange(0, P, P // 8), P // 2 + np.arange(-4, 4),
                                     np.random.default_rng(N).integers(0, P, 8)]))
    Ig = I[:, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    for j, lam in enumerate(lams[:1] if N == 8192 else lams):
        ref = oracle.psf_rows(h, dx, z, lam, rows)
        err = rel_l2(Ig[j], ref)
        assert err < TOL_PSF, (j, err)
    # Parseval over the band on every wavelength: sum I <= N^2 and close to it for smooth h
    tot = I.double().sum(dim=(1, 2)).cpu().numpy()
    assert np.all(tot <= N * N * (1 + 1e-5)) and np.all(tot > 0.5 * N * N)


def test_band_mask_bit_exact():
    # power-of-two grids and mixed-radix ones (P = 360, 3600: the same integer band logic)
    for N, dx, z, lams in [(32, 0.25e-6, 5e-6, [400e-9, 700e-9]), (256, 2e-6, 20e-3, [550e-9]),
                           (512, 1e-6, 50e-3, [450e-9, 650e-9]), (180, 1e-6, 2e-3, [500e-9]),
                           (1800, 2e-6, 10e-3, [520.6e-9])]:
        g = Geometry.make(N, dx, z, lams)
        for j, lam in enumerate(lams):
            m = api.debug_band_mask(g, j).cpu().numpy()
            ref = oracle.band_mask(2 * N, dx, z, lam)
            assert np.array_equal(m, ref)


def test_deterministic_and_batch_invariant():
    N, dx, z = 256, 1e-6, 5e-3
    h1 = torch.from_numpy(_h(N, 3)).cuda()
    h2 = torch.from_numpy(_h(N, 4)).cuda()
    g1 = Geometry.make(N, dx, z, [450e-9, 600e-9])
    g2 = Geometry.make(N, dx, 2 * z, [700e-9])
    a = api.psf(h1, g1)
    b = api.psf(h1, g1)
    assert torch.equal(a, b)
    many = api.psf_many([h1, h2], [g1, g2])
    assert torch.equal(many[0], a)
    assert torch.equal(many[1], api.psf(h2, g2))


# -------------------------------------------------------------- gradient
def test_grad_matches_oracle_512():
    # 256 x 256 DOE, 3 wavelengths, padded 512 x 512: full FP64 oracle gradient
    N, dx, z = 256, 2e-6, 20e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = 2 * N
    h = _h(N, 1001)
    T = inputs.spot_target(P, N, 3, 2003)
    g = Geometry.make(N, dx, z, lams)
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    ref, ref_loss = oracle.grad(h, dx, z, lams, T)
    err = rel_l2(gr.cpu().numpy(), ref)
    assert err < TOL_GRAD, err
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss


def test_grad_vjp_and_autograd():
    N, dx, z = 128, 1e-6, 3e-3
    lams = [500e-9, 620e-9]
    P = 2 * N
    h = _h(N, 9)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((2, P, P)).astype(np.float32)
    g = Geometry.make(N, dx, z, lams)
    ht = torch.from_numpy(h).cuda().requires_grad_(True)
    I = api.psf_autograd(ht, g)
    I.backward(torch.from_numpy(G).cuda())
    ref, _ = oracle.grad(h, dx, z, lams, G, mode="vjp")
    assert rel_l2(ht.grad.cpu().numpy(), ref) < TOL_GRAD


def test_grad_stored_fields_equal_recompute():
    N, dx, z = 256, 1e-6, 5e-3
    lams = [450e-9, 650e-9]
    P = 2 * N
    h = torch.from_numpy(_h(N, 12)).cuda()
    T = torch.from_numpy(inputs.spot_target(P, N, 2, 2012)).cuda()
    g = Geometry.make(N, dx, z, lams)
    ws = api.workspace(api.workspace_bytes(g, 3))
    a, la = api.grad(h, g, T, ws=ws, recompute=True)
    api.psf(h, g, ws=ws)
    b, lb = api.grad(h, g, T, ws=ws, recompute=False)
    assert torch.equal(a, b) and torch.equal(la, lb)


def test_grad_finite_differences_fd_exact():
    # central differences of the FP64 loss (exact-difference form) on seeded pixels
    N, dx, z = 512, 1e-6, 10e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = 2 * N
    h = _h(N, 31)
    T = inputs.spot_target(P, N, 3, 2031)
    g = Geometry.make(N, dx, z, lams)
    gr, _ = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    gr = gr.cpu().numpy()
    rng = np.random.default_rng(64)
    py = rng.integers(0, N, 16)
    px = rng.integers(0, N, 16)
    fd = oracle.fd_exact(h, dx, z, lams, T, py, px, 1e-10)
    scale = np.abs(fd).max()
    assert np.all(np.abs(gr[py, px] - fd) <= 1e-3 * scale), np.abs(gr[py, px] - fd).max() / scale


# -------------------------------------------------------------- render
@pytest.mark.parametrize("C,H,W,Pp", [(2, 16, 32, 64), (3, 64, 64, 128), (1, 128, 256, 512)])
def test_render_small_vs_oracle(C, H, W, Pp):
    rng = np.random.default_rng(H + W)
    psf = rng.random((C, Pp, Pp)).astype(np.float32) ** 4
    img = inputs.image(C, H, W, 2000 + H)
    out = api.render(torch.from_numpy(psf).cuda(), torch.from_numpy(img).cuda()).cpu().numpy()
    ref = oracle.render(psf, img)
    assert rel_l2(out, ref) < TOL_PSF, rel_l2(out, ref)


def _rgb_workload_psfs():
    # the oracle's FP64 PSFs of the RGB workload's 4096^2 DOE (8192^2 grid, 450/550/650 nm),
    # rounded to float32: the input both sides of the render and Wiener tests receive
    N, dx, z = 4096, 1e-6, 50e-3
    return oracle.psf(_h(N, 1002), dx, z, [450e-9, 550e-9, 650e-9]).astype(np.float32)


def test_render_rgb_workload_vs_oracle():
    # the RGB design-evaluation workload: 3 PSFs of a 4096^2 DOE (8192^2 grid) convolved with
    # a seeded 3 x 2048 x 2048 scene
    psf = _rgb_workload_psfs()
    img = inputs.image(3, 2048, 2048, 2002)
    out = api.render(torch.from_numpy(psf).cuda(), torch.from_numpy(img).cuda()).cpu().numpy()
    ref = oracle.render(psf, img)
    assert rel_l2(out, ref) < TOL_PSF, rel_l2(out, ref)


# -------------------------------------------------------------- Wiener deconvolution (Eq. 9)
GAMMA = 5e-4  # the regulariser of the imaging application
# FP32 transforms (rel L2 <= TOL_PSF, as for the PSF) amplified by at most the filter's gain
# max |conj(K) / (|K|^2 + gamma)| = 1 / (2 sqrt(gamma))
TOL_WIENER = TOL_PSF / (2.0 * np.sqrt(GAMMA))


@pytest.mark.parametrize("C,H,W,Pp", [(2, 32, 32, 64), (3, 64, 128, 128), (1, 256, 64, 512)])
def test_wiener_small_vs_oracle(C, H, W, Pp):
    rng = np.random.default_rng(7 * H + W)
    psf = rng.random((C, Pp, Pp)).astype(np.float32) ** 4
    y = inputs.image(C, H, W, 2100 + H)
    out = api.wiener(torch.from_numpy(psf).cuda(), torch.from_numpy(y).cuda(), GAMMA).cpu().numpy()
    ref = oracle.wiener(psf, y, GAMMA)
    assert rel_l2(out, ref) < TOL_WIENER, rel_l2(out, ref)


def test_wiener_rgb_workload_vs_oracle():
    # the RGB workload's PSFs deconvolving a scene the oracle blurred with them
    psf = _rgb_workload_psfs()
    y = oracle.render(psf, inputs.image(3, 2048, 2048, 2002)).astype(np.float32)
    out = api.wiener(torch.from_numpy(psf).cuda(), torch.from_numpy(y).cuda(), GAMMA).cpu().numpy()
    ref = oracle.wiener(psf, y, GAMMA)
    err = rel_l2(out, ref)
    print(f"wiener rgb rel_l2 {err:.3e}")
    assert err < TOL_WIENER, err


def test_wiener_rejects_bad_arguments():
    psf = torch.zeros((1, 64, 66), device="cuda")  # Px not a multiple of 4
    y = torch.zeros((1, 32, 32), device="cuda")
    with pytest.raises(Exception):
        api.wiener(psf, y, GAMMA)
    with pytest.raises(Exception):
        api.wiener(torch.zeros((1, 64, 64), device="cuda"), y, -1.0)


def test_trace_and_launch_count():
    N = 256
    h = torch.from_numpy(_h(N, 5)).cuda()
    g = Geometry.make(N, 1e-6, 5e-3, [500e-9])
    api.psf(h, g)
    n0 = api.launch_count()
    api.trace_enable(16)
    api.psf(h, g)
    recs = api.trace_read()
    api.trace_enable(0)
    assert [r[0] for r in recs] == ["transfer_table", "pass_a_rows", "pass_b_columns", "pass_c_rows"]
    assert all(ms > 0 for _, ms in recs)
    assert api.launch_count() - n0 == 4


# -------------------------------------------------------------- grids longer than one CTA
def _h_closed(kt, lt, P, dx, z, lam):
    """Transfer function at integer frequencies, FP64, from its definition (band + evanescent
    rules as stated for the oracle)."""
    du = 1.0 / (P * dx)
    kmax = oracle.kmax(lam, dx, P, z)
    if abs(kt) > kmax or abs(lt) > kmax or kt * kt + lt * lt >= oracle.m_ev(lam, dx, P):
        return 0.0
    ph = 2 * np.pi * z * np.sqrt(1.0 / lam**2 - (kt * du) ** 2 - (lt * du) ** 2)
    return np.exp(1j * np.fmod(ph, 2 * np.pi))


@pytest.mark.parametrize("P", [32768, 65536])
def test_big_grid_flat_plate(P):
    c, dx, z, lam = 0.37e-6, 1e-6, 0.1, 550e-9
    h = torch.full((P, P), c, dtype=torch.float32, device="cuda")
    g = Geometry.make(P, dx, z, [lam], pad=1)
    e = api.propagate(h, g)[0]
    phase = 2 * np.pi * 0.46 * float(np.float32(c)) / lam + 2 * np.pi * z / lam
    ref = torch.tensor(complex(np.cos(np.fmod(phase, 2 * np.pi)), np.sin(np.fmod(phase, 2 * np.pi))),
                       dtype=torch.complex64, device="cuda")
    err = (e - ref).abs().max().item()
    assert err < 5e-5, err


def test_big_grid_plane_waves_closed_form():
    # pad 1, h = 0, E_in = sum_j c_j exp(2 pi i (a_j x + b_j y) / P): every wave is a single
    # spectral line, so E_out = sum_j c_j H(a_j, b_j) exp(2 pi i (a_j x + b_j y) / P)
    P, dx, z, lam = 65536, 1e-6, 0.1, 550e-9
    rng = np.random.default_rng(65536)
    waves = [(int(a), int(b), complex(rng.standard_normal(), rng.standard_normal()))
             for a, b in rng.integers(-P // 2, P // 2, size=(6, 2))] + [(0, 0, 1.0 + 0.5j), (P // 2 - 1, -3, 0.7 - 0.2j)]
    ys = torch.arange(P, device="cuda", dtype=torch.float64)

    def field(coefs, rows=None):
        yy = ys if rows is None else rows
        out = torch.zeros((yy.numel(), P), dtype=torch.complex128, device="cuda")
        for (a, b, _), cc in zip(waves, coefs):
            px = torch.exp(2j * np.pi * ((a * ys) % P) / P)
            py = torch.exp(2j * np.pi * ((b * yy) % P) / P)
            out += cc * py[:, None] * px[None, :]
        return out

    e_in = torch.empty((P, P), dtype=torch.complex64, device="cuda")
    for r0 in range(0, P, 4096):
        e_in[r0:r0 + 4096] = field([w[2] for w in waves], ys[r0:r0 + 4096]).to(torch.complex64)
    g = Geometry.make(P, dx, z, [lam], pad=1)
    e = api.propagate(torch.zeros((P, P), dtype=torch.float32, device="cuda"), g, e_in=e_in)[0]
    del e_in
    rows = torch.tensor([0, 1, 777, P // 2, P - 1], device="cuda", dtype=torch.float64)
    ref = field([w[2] * _h_closed(w[0], w[1], P, dx, z, lam) for w in waves], rows)
    got = e[rows.long()].to(torch.complex128)
    err = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
    assert err < TOL_PSF, err


def test_big_grid_psf_rows_vs_oracle():
    # 16384 x 16384 DOE padded to 32768 x 32768 (two-CTA rows and columns)
    N, dx, z, lam = 16384, 1e-6, 50e-3, 550e-9
    P = 2 * N
    h = _h(N, 1005)
    g = Geometry.make(N, dx, z, [lam])
    I = api.psf(torch.from_numpy(h).cuda(), g)
    rows = np.array([0, P // 4, P // 2 - 1, P // 2, P // 2 + 3, 3 * P // 4, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    ref = oracle.psf_rows(h, dx, z, lam, rows)
    err = rel_l2(Ig, ref)
    assert err < TOL_PSF, err


def test_large_area_psf_rows_vs_oracle():
    # the large-area workload: 32768 x 32768 DOE at 1 um, 550 nm, z = 100 mm, padded to
    # 65536 x 65536 (band limit inactive); exact FP64 rows from the oracle's row-subset mode
    N, dx, z, lam = 32768, 1e-6, 100e-3, 550e-9
    P = 2 * N
    h = _h(N, 1004)
    g = Geometry.make(N, dx, z, [lam])
    I = api.psf(torch.from_numpy(h).cuda(), g)
    rows = np.array([0, P // 8, P // 2 - 1, P // 2, 5 * P // 8, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    tot = I.double().sum().item()
    del I
    ref = oracle.psf_rows(h, dx, z, lam, rows)
    err = rel_l2(Ig, ref)
    assert err < TOL_PSF, err
    assert 0.5 * N * N < tot <= N * N * (1 + 1e-5)  # Parseval over the band


def test_large_area_gradient_rows_vs_oracle():
    # the large-area gradient (32768^2 DOE, 65536^2 grid, adjoint with recomputed fields): a
    # vector-Jacobian product whose dL/dI is non-zero on seeded output rows only, against the
    # oracle's row-subset adjoint on seeded DOE rows (the FP64 field does not fit host memory)
    N, dx, z, lam = 32768, 1e-6, 100e-3, 550e-9
    P = 2 * N
    h = _h(N, 1004)
    g = Geometry.make(N, dx, z, [lam])
    r = np.random.default_rng(4004)
    rows = np.unique(np.concatenate([[P // 4, P // 2, P // 2 + 1, 3 * P // 4 - 1, P - 1], r.integers(0, P, 11)]))
    g_rows = r.standard_normal((rows.size, P)).astype(np.float32)
    G = torch.zeros((1, P, P), dtype=torch.float32, device="cuda")
    G[0, torch.from_numpy(rows).cuda()] = torch.from_numpy(g_rows).cuda()
    gr, _ = api.grad(torch.from_numpy(h).cuda(), g, G, mode="vjp", recompute=True)
    drows = np.unique(np.concatenate([[0, N // 2, N - 1], r.integers(0, N, 13)]))
    got = gr[torch.from_numpy(drows).cuda()].cpu().numpy()
    del G, gr
    torch.cuda.empty_cache()
    ref = oracle.grad_rows(h, dx, z, lam, rows, g_rows, drows)
    err = rel_l2(got, ref)
    assert err < TOL_GRAD, err


def test_big_grid_gradient_fd_exact():
    # two-CTA rows/columns adjoint (16384^2 DOE, 32768^2 grid) against exact-difference
    # central differences of the FP64 loss on seeded pixels
    N, dx, z = 16384, 1e-6, 50e-3
    lams = [550e-9]
    P = 2 * N
    h = _h(N, 1006)
    T = inputs.spot_target(P, N, 1, 2006)
    g = Geometry.make(N, dx, z, lams)
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    gr = gr.cpu().numpy()
    rng = np.random.default_rng(16384)
    py = np.concatenate([rng.integers(0, N, 6), [N // 2, N // 2 + 1]])
    px = np.concatenate([rng.integers(0, N, 6), [N // 2, N // 2]])
    fd = oracle.fd_exact(h, dx, z, lams, T, py, px, 1e-10)
    scale = np.abs(fd).max()
    assert np.all(np.abs(gr[py, px] - fd) <= 1e-3 * scale), np.abs(gr[py, px] - fd).max() / scale


def test_gradient_workload_fd_exact():
    # the gradient workload: 8192 x 8192 DOE, 3 wavelengths, padded 16384 x 16384, spot-array
    # target; central differences (step 1e-4 um) of the FP64 loss on 64 seeded pixels
    N, dx, z = 8192, 1e-6, 50e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = 2 * N
    h = _h(N, 1003)
    T = inputs.spot_target(P, N, 3, 2003)
    g = Geometry.make(N, dx, z, lams)
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    gr = gr.cpu().numpy()
    rng = np.random.default_rng(8192)
    py = rng.integers(0, N, 64)  # 64 seeded pixels
    px = rng.integers(0, N, 64)
    fd = oracle.fd_exact(h, dx, z, lams, T, py, px, 1e-10)
    scale = np.abs(fd).max()
    assert np.all(np.abs(gr[py, px] - fd) <= 1e-3 * scale), np.abs(gr[py, px] - fd).max() / scale


# -------------------------------------------------------------- super-resolved design input
@pytest.mark.parametrize("N,f,pad", [(256, 2, 2), (256, 4, 2), (256, 8, 2), (128, 4, 1)])
def test_upsampled_layout_psf_and_grad_vs_oracle(N, f, pad):
    # heights on an (N / f)^2 layout at pitch f dx, nearest-upsampled inside the first pass;
    # the oracle gets the upsampled heights and returns the layout gradient as block sums
    dx, z = 0.5e-6, 2e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = pad * N
    hl = _h(N // f, 5000 + f)
    g = Geometry.make(N, dx, z, lams, pad=pad, upsample=f)
    hs = oracle.upsample_nearest(hl, f)
    I = api.psf(torch.from_numpy(hl).cuda(), g).cpu().numpy()
    ref = oracle.psf(hs, dx, z, lams, pad=pad)
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    T = inputs.spot_target(P, N, 3, 6000 + f)
    gr, loss = api.grad(torch.from_numpy(hl).cuda(), g, torch.from_numpy(T).cuda())
    assert gr.shape == (N // f, N // f)
    gref, lref = oracle.grad(hs, dx, z, lams, T, pad=pad)
    err = rel_l2(gr.cpu().numpy(), oracle.layout_grad(gref, f))
    assert err < TOL_GRAD, err
    assert abs(loss.item() - lref) <= 1e-5 * lref


def test_upsampled_layout_big_grid_rows_vs_oracle():
    # 4096^2 layout, 4x nearest upsampling onto a 16384^2 DOE, 32768^2 grid (cluster-split rows)
    N, f, dx, z, lam = 16384, 4, 0.5e-6, 20e-3, 550e-9
    P = 2 * N
    hl = _h(N // f, 5100)
    g = Geometry.make(N, dx, z, [lam], upsample=f)
    I = api.psf(torch.from_numpy(hl).cuda(), g)
    rows = np.array([0, P // 4, P // 2 - 1, P // 2, 3 * P // 4 + 5, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    del I
    ref = oracle.psf_rows(oracle.upsample_nearest(hl, f), dx, z, lam, rows)
    err = rel_l2(Ig, ref)
    assert err < TOL_PSF, err


def test_upsampled_and_plain_requests_share_a_launch():
    N, dx, z = 256, 0.5e-6, 2e-3
    h1 = torch.from_numpy(_h(N, 5200)).cuda()
    h2 = torch.from_numpy(_h(N // 4, 5201)).cuda()
    g1 = Geometry.make(N, dx, z, [500e-9])
    g2 = Geometry.make(N, dx, z, [600e-9, 700e-9], upsample=4)
    many = api.psf_many([h1, h2], [g1, g2])
    assert torch.equal(many[0], api.psf(h1, g1))
    assert torch.equal(many[1], api.psf(h2, g2))


@pytest.mark.parametrize("N,f,pad", [(256, 2, 2), (256, 4, 2), (256, 8, 2), (128, 4, 1)])
def test_lanczos_layout_psf_and_grad_vs_oracle(N, f, pad):
    # Lanczos-3 interpolation of an (N / f)^2 layout (a pre-pass), then the PSF and the layout
    # gradient (the transpose of the interpolation applied to the grid gradient)
    dx, z = 0.5e-6, 2e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = pad * N
    hl = _h(N // f, 5300 + f)
    g = Geometry.make(N, dx, z, lams, pad=pad, upsample=f, lanczos=True)
    hs = oracle.upsample_lanczos3(hl, f)
    I = api.psf(torch.from_numpy(hl).cuda(), g).cpu().numpy()
    ref = oracle.psf(hs, dx, z, lams, pad=pad)
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    T = inputs.spot_target(P, N, 3, 6300 + f)
    for recompute in (True, False):
        if not recompute:
            ws = api.workspace(api.workspace_bytes(g, 3))  # gradient-sized: the PSF call keeps its fields
            api.psf(torch.from_numpy(hl).cuda(), g, ws=ws)
        else:
            ws = None
        gr, loss = api.grad(torch.from_numpy(hl).cuda(), g, torch.from_numpy(T).cuda(), recompute=recompute, ws=ws)
        assert gr.shape == (N // f, N // f)
        gref, lref = oracle.grad(hs, dx, z, lams, T, pad=pad)
        err = rel_l2(gr.cpu().numpy(), oracle.layout_grad_lanczos3(gref, f))
        assert err < TOL_GRAD, err
        assert abs(loss.item() - lref) <= 1e-5 * lref


def test_lanczos_layout_rows_at_4096_vs_oracle():
    # 1024^2 layout, Lanczos-3 by 4 onto a 4096^2 DOE, 8192^2 grid: sampled output rows
    N, f, dx, z, lam = 4096, 4, 0.5e-6, 5e-3, 550e-9
    P = 2 * N
    hl = _h(N // f, 5400)
    g = Geometry.make(N, dx, z, [lam], upsample=f, lanczos=True)
    I = api.psf(torch.from_numpy(hl).cuda(), g)
    rows = np.array([0, P // 4, P // 2 - 1, P // 2, 3 * P // 4 + 5, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    ref = oracle.psf_rows(oracle.upsample_lanczos3(hl, f), dx, z, lam, rows)
    err = rel_l2(Ig, ref)
    assert err < TOL_PSF, err


def test_lanczos_nearest_and_plain_requests_share_a_launch():
    N, dx, z = 256, 0.5e-6, 2e-3
    h1 = torch.from_numpy(_h(N, 5500)).cuda()
    h2 = torch.from_numpy(_h(N // 4, 5501)).cuda()
    h3 = torch.from_numpy(_h(N // 2, 5502)).cuda()
    h4 = torch.from_numpy(_h(N // 8, 5503)).cuda()
    gs = [Geometry.make(N, dx, z, [500e-9]),
          Geometry.make(N, dx, z, [600e-9, 700e-9], upsample=4, lanczos=True),
          Geometry.make(N, dx, z, [450e-9], upsample=2),
          Geometry.make(N, dx, z, [550e-9, 650e-9], upsample=8, lanczos=True)]
    many = api.psf_many([h1, h2, h3, h4], gs)
    for h, g, m in zip([h1, h2, h3, h4], gs, many):
        assert torch.equal(m, api.psf(h, g))


# -------------------------------------------------------------- parametric incident fields
ILLUM_CASES = {
    "tilt": dict(theta_x=0.1, theta_y=-0.05),
    "converging": dict(src_d=-2e-3),
    "diverging": dict(src_d=5e-3),
    "tilted_converging": dict(theta_x=-0.08, theta_y=0.03, src_d=-3e-3),
}


def _illum_oracle(hs, N, dx, z, lams, kw, T=None, pad=2, e_arr=None):
    """Per-wavelength oracle PSFs (and the gradient summed over wavelengths) with E_in the
    oracle's incident field of each wavelength, times e_arr if given."""
    I, g, loss = [], 0.0, 0.0
    for j, lam in enumerate(lams):
        e = oracle.incident(N, dx, lam, kw.get("theta_x", 0.0), kw.get("theta_y", 0.0), kw.get("src_d", 0.0))
        if e_arr is not None:
            e = e * e_arr
        I.append(oracle.psf(hs, dx, z, [lam], pad=pad, e_in=e)[0])
        if T is not None:
            gj, lj = oracle.grad(hs, dx, z, [lam], T[j:j + 1], pad=pad, e_in=e)
            g, loss = g + gj, loss + lj
    return np.stack(I), g, loss


@pytest.mark.parametrize("case", sorted(ILLUM_CASES))
@pytest.mark.parametrize("N,pad", [(256, 2), (128, 1)])
def test_incident_field_psf_and_grad_vs_oracle(case, N, pad):
    dx, z = 0.5e-6, 2e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = pad * N
    kw = ILLUM_CASES[case]
    h = _h(N, 8000 + N)
    T = inputs.spot_target(P, N, 3, 8100 + N)
    g = Geometry.make(N, dx, z, lams, pad=pad, **kw)
    I = api.psf(torch.from_numpy(h).cuda(), g).cpu().numpy()
    gr, loss = api.grad(torch.from_numpy(h).cuda(), g, torch.from_numpy(T).cuda())
    Iref, gref, lref = _illum_oracle(h, N, dx, z, lams, kw, T, pad=pad)
    assert rel_l2(I, Iref) < TOL_PSF, rel_l2(I, Iref)
    err = rel_l2(gr.cpu().numpy(), gref)
    assert err < TOL_GRAD, err
    assert abs(loss.item() - lref) <= 1e-5 * lref


def test_incident_field_with_array_and_upsampling_vs_oracle():
    # the parametric field multiplies an E_in array; heights on a 4x nearest-upsampled layout
    N, f, dx, z = 256, 4, 0.5e-6, 2e-3
    lams = [500e-9, 620e-9]
    kw = dict(theta_x=0.06, src_d=-4e-3)
    hl = _h(N // f, 8200)
    hs = oracle.upsample_nearest(hl, f)
    e_arr = inputs.gaussian_beam(N, dx, 40e-6).astype(np.complex64)
    T = inputs.spot_target(2 * N, N, 2, 8201)
    g = Geometry.make(N, dx, z, lams, upsample=f, **kw)
    et = torch.from_numpy(e_arr).cuda()
    I = api.psf(torch.from_numpy(hl).cuda(), g, e_in=et).cpu().numpy()
    gr, loss = api.grad(torch.from_numpy(hl).cuda(), g, torch.from_numpy(T).cuda(), e_in=et)
    Iref, gref, lref = _illum_oracle(hs, N, dx, z, lams, kw, T, e_arr=e_arr.astype(np.complex128))
    assert rel_l2(I, Iref) < TOL_PSF, rel_l2(I, Iref)
    err = rel_l2(gr.cpu().numpy(), oracle.layout_grad(gref, f))
    assert err < TOL_GRAD, err
    assert abs(loss.item() - lref) <= 1e-5 * lref


def test_incident_field_requests_share_a_launch():
    # tilted, spherical and plain requests in one batched launch equal their separate calls
    N, dx, z = 256, 0.5e-6, 2e-3
    hs = [torch.from_numpy(_h(N, 8300 + k)).cuda() for k in range(3)]
    gs = [Geometry.make(N, dx, z, [500e-9]),
          Geometry.make(N, dx, z, [600e-9, 700e-9], theta_x=0.05),
          Geometry.make(N, dx, z, [450e-9], src_d=-2e-3)]
    many = api.psf_many(hs, gs)
    for h, g, m in zip(hs, gs, many):
        assert torch.equal(m, api.psf(h, g))


def test_incident_field_big_grid_rows_vs_oracle():
    # 16384^2 DOE, 32768^2 grid (cluster-split rows): a tilted wave converging to 200 mm,
    # sampled PSF rows and the row-subset gradient against the oracle
    N, dx, z, lam = 16384, 1e-6, 50e-3, 550e-9
    P = 2 * N
    kw = dict(theta_x=0.01, theta_y=-0.005, src_d=-0.2)
    h = _h(N, 8400)
    g = Geometry.make(N, dx, z, [lam], **kw)
    e = oracle.incident(N, dx, lam, theta_x=0.01, theta_y=-0.005, d=-0.2)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g)
    rows = np.array([0, P // 4, P // 2 - 1, P // 2, 3 * P // 4 + 5, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    del I
    err = rel_l2(Ig, oracle.psf_rows(h, dx, z, lam, rows, e_in=e))
    assert err < TOL_PSF, err
    r = np.random.default_rng(8401)
    grows = np.unique(np.concatenate([[P // 2, P // 2 + 1], r.integers(0, P, 6)]))
    g_rows = r.standard_normal((grows.size, P)).astype(np.float32)
    G = torch.zeros((1, P, P), dtype=torch.float32, device="cuda")
    G[0, torch.from_numpy(grows).cuda()] = torch.from_numpy(g_rows).cuda()
    gr, _ = api.grad(ht, g, G, mode="vjp", recompute=True)
    drows = np.unique(np.concatenate([[0, N // 2, N - 1], r.integers(0, N, 5)]))
    got = gr[torch.from_numpy(drows).cuda()].cpu().numpy()
    del G, gr
    torch.cuda.empty_cache()
    err = rel_l2(got, oracle.grad_rows(h, dx, z, lam, grows, g_rows, drows, e_in=e))
    assert err < TOL_GRAD, err


# -------------------------------------------------------------- design optimiser
def test_adam_step_matches_oracle():
    r = np.random.default_rng(50)
    n = 4096
    h0 = (r.random(n) * 1.2e-6).astype(np.float32)
    ht, mt, vt = torch.from_numpy(h0).cuda(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    ho, mo, vo = h0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 7):
        g = (r.standard_normal(n) * 1e3).astype(np.float32)
        api.adam_step(ht, torch.from_numpy(g).cuda(), mt, vt, 2e-8, t, h_max=1.2e-6)
        ho, mo, vo = oracle.adam_step(ho, g, mo, vo, 2e-8, t, h_max=1.2e-6)
    assert rel_l2(ht.cpu().numpy(), ho) < 1e-6


@pytest.mark.parametrize("target", ["spots", "flat_top"])
def test_design_loop_matches_oracle(target):
    # Adam + cosine schedule on the L2 gradient (64^2 DOE, 2 wavelengths, 6 steps), the GPU
    # library against the same loop on the FP64 oracle's gradient and Adam; targets: the
    # Gaussian spot lattice and the flat-top 8 x 8 beam-splitter lattice
    from paper_2505_22313_b300 import design

    N, dx, z = 64, 1e-6, 2e-3
    lams = [500e-9, 600e-9]
    P = 2 * N
    iters, lr0 = 6, 1.2e-8
    h0 = _h(N, 7000)
    T = inputs.spot_target(P, N, 2, 7001) if target == "spots" else inputs.flat_top_target(P, N, 2)
    g = Geometry.make(N, dx, z, lams)
    h, losses = design.optimize(torch.from_numpy(h0).cuda(), g, torch.from_numpy(T).cuda(), iters, lr0=lr0)
    ho, mo, vo = h0.astype(np.float64), np.zeros((N, N)), np.zeros((N, N))
    lo = []
    for t in range(1, iters + 1):
        gr, loss = oracle.grad(ho.astype(np.float32), dx, z, lams, T)
        lo.append(loss)
        ho, mo, vo = oracle.adam_step(ho, gr, mo, vo, oracle.cosine_lr(lr0, t, iters), t, h_max=inputs.HMAX)
    lg = losses.cpu().numpy()
    assert np.all(np.abs(lg - np.array(lo)) <= 1e-4 * np.abs(lo)), (lg, lo)
    assert lo[-1] < lo[0]  # the loop descends
    assert rel_l2(h.cpu().numpy(), ho) < 1e-3


# -------------------------------------------------------------- radial parameterisation
@pytest.mark.parametrize("n,n_c", [(16, 1), (256, 5), (256, 9), (4096, 9), (1800, 9), (20000, 9)])
def test_radial_heights_vs_oracle(n, n_c):
    r = np.random.default_rng(9000 + n_c)
    c = (r.standard_normal(n_c) * 3e-7).astype(np.float32)
    h = api.radial_heights(torch.from_numpy(c).cuda(), n).cpu().numpy()
    ref = oracle.radial_heights(c.astype(np.float64), n)
    # double-float Horner then one rounding: within an ulp of the exact value
    assert np.all(np.abs(h - ref) <= 2.0**-23 * np.abs(ref) + 1e-12 * np.abs(c).sum())


@pytest.mark.parametrize("n", [64, 2048, 1800])
def test_radial_grad_vs_oracle(n):
    r = np.random.default_rng(9100 + n)
    g = r.standard_normal((n, n)).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    got = api.radial_grad(gt, 9).cpu().numpy()
    ref = oracle.radial_grad(g, 9)
    s = oracle.radial_s(n)
    scale = np.array([(np.abs(g.astype(np.float64)) * s**k).sum() for k in range(9)])
    # float32 rounding of each result, and FP64-level summation of the terms
    assert np.all(np.abs(got - ref) <= 2.0**-23 * np.abs(ref) + 1e-12 * scale), (got, ref)
    assert torch.equal(api.radial_grad(gt, 9), api.radial_grad(gt, 9))  # fixed summation order


def test_radial_design_loop_matches_oracle():
    # radially symmetric design (Sec. 5.4): Adam on 9 even-polynomial coefficients towards an
    # on-axis focus, 64^2 DOE, 2 wavelengths, 5 steps, against the same loop on the oracle
    from paper_2505_22313_b300 import design

    N, dx, z = 64, 1e-6, 2e-3
    lams = [500e-9, 600e-9]
    P = 2 * N
    iters, lr0 = 5, 3e-9
    c0 = np.zeros(9, np.float32)
    c0[0], c0[1] = 0.6e-6, -0.3e-6
    T = inputs.spot_target(P, N, 2, 9201, grid=1)
    g = Geometry.make(N, dx, z, lams)
    c, losses = design.optimize_radial(torch.from_numpy(c0).cuda(), g, torch.from_numpy(T).cuda(), iters, lr0)
    co, mo, vo = c0.astype(np.float64), np.zeros(9), np.zeros(9)
    lo = []
    inf = np.inf
    for t in range(1, iters + 1):
        h = oracle.radial_heights(co.astype(np.float32).astype(np.float64), N).astype(np.float32)
        gh, loss = oracle.grad(h, dx, z, lams, T)
        lo.append(loss)
        gc = oracle.radial_grad(gh, 9)
        co, mo, vo = oracle.adam_step(co, gc, mo, vo, oracle.cosine_lr(lr0, t, iters), t, h_min=-inf, h_max=inf)
    lg = losses.cpu().numpy()
    assert np.all(np.abs(lg - np.array(lo)) <= 1e-4 * np.abs(lo)), (lg, lo)
    assert lo[-1] < lo[0]
    cg = c.cpu().numpy()
    # the piston c[0] has a zero gradient (a global phase), so Adam moves it by the sign of
    # rounding noise: compare it only up to the steps taken
    assert rel_l2(cg[1:], co[1:]) < 1e-3
    assert abs(cg[0] - co[0]) <= iters * lr0


# -------------------------------------------------------------- non-power-of-two grids
@pytest.mark.parametrize("N,pad", [(24, 2), (90, 2), (180, 2), (360, 1), (1500, 2), (90, 1), (150, 1)])
def test_mixed_radix_propagate_vs_oracle(N, pad):
    # P = 48, 180, 360, 360, 3000: radix 2, 3, 4, 5, 8 stages; P = 90, 150 (not multiples of 4):
    # the column pass without clusters
    dx, z, lam = 1e-6, 2e-3, 550e-9
    h = _h(N, 9500 + N)
    g = Geometry.make(N, dx, z, [lam], pad=pad)
    E = api.propagate(torch.from_numpy(h).cuda(), g).cpu().numpy()[0]
    ref = oracle.propagate(h, dx, z, lam, pad=pad)
    assert rel_l2(E, ref) < TOL_PSF, rel_l2(E, ref)


@pytest.mark.parametrize("N,pad,bandlimit", [(180, 2, True), (360, 1, True), (180, 2, False)])
def test_mixed_radix_psf_and_grad_vs_oracle(N, pad, bandlimit):
    dx, z = 0.5e-6, 2e-3
    lams = [450e-9, 550e-9, 650e-9]
    P = pad * N
    h = _h(N, 9600 + N)
    T = inputs.spot_target(P, N, 3, 9700 + N)
    g = Geometry.make(N, dx, z, lams, pad=pad, bandlimit=bandlimit)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    ref = oracle.psf(h, dx, z, lams, pad=pad, bandlimit=bandlimit)
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    gref, lref = oracle.grad(h, dx, z, lams, T, pad=pad, bandlimit=bandlimit)
    for recompute in (True, False):
        ws = None
        if not recompute:
            ws = api.workspace(api.workspace_bytes(g, 3))
            api.psf(ht, g, ws=ws)
        gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda(), recompute=recompute, ws=ws)
        err = rel_l2(gr.cpu().numpy(), gref)
        assert err < TOL_GRAD, err
        assert abs(loss.item() - lref) <= 1e-5 * lref


def test_mixed_radix_table2_grid_3600():
    # Table 2's first grid: a 3.6 mm DOE at 2 um (1800^2), padded to 3600 x 3600, 520.6 nm
    # laser (Sec. 3.2's toy example), hologram plane at 10 mm: PSF and L2 gradient vs the oracle
    N, dx, z, lam = 1800, 2e-6, 10e-3, 520.6e-9
    P = 2 * N
    h = _h(N, 9800)
    T = inputs.flat_top_target(P, N, 1)
    g = Geometry.make(N, dx, z, [lam])
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    assert rel_l2(I, oracle.psf(h, dx, z, [lam])) < TOL_PSF
    gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad(h, dx, z, [lam], T)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref


def test_mixed_radix_with_upsampling_illumination_and_batching():
    # 45^2 layout, 4x nearest-upsampled onto a 180^2 DOE, 360^2 grid, tilted converging wave;
    # Lanczos-3 variant; and three requests of one grid in one batched launch
    N, f, dx, z = 180, 4, 0.5e-6, 2e-3
    lams = [500e-9, 620e-9]
    kw = dict(theta_x=0.05, src_d=-3e-3)
    hl = _h(N // f, 9900)
    T = inputs.spot_target(2 * N, N, 2, 9901)
    for lanczos in (False, True):
        hs = oracle.upsample_lanczos3(hl, f) if lanczos else oracle.upsample_nearest(hl, f)
        g = Geometry.make(N, dx, z, lams, upsample=f, lanczos=lanczos, **kw)
        I = api.psf(torch.from_numpy(hl).cuda(), g).cpu().numpy()
        gr, loss = api.grad(torch.from_numpy(hl).cuda(), g, torch.from_numpy(T).cuda())
        Iref, gref, lref = _illum_oracle(hs, N, dx, z, lams, kw, T)
        assert rel_l2(I, Iref) < TOL_PSF, rel_l2(I, Iref)
        lg = oracle.layout_grad_lanczos3(gref, f) if lanczos else oracle.layout_grad(gref, f)
        assert rel_l2(gr.cpu().numpy(), lg) < TOL_GRAD
        assert abs(loss.item() - lref) <= 1e-5 * lref
    hs3 = [torch.from_numpy(_h(N, 9910 + k)).cuda() for k in range(3)]
    gs = [Geometry.make(N, dx, z, [500e-9]), Geometry.make(N, dx, 3e-3, [600e-9, 700e-9]),
          Geometry.make(N, dx, z, [450e-9], theta_y=0.02)]
    for h, gg, m in zip(hs3, gs, api.psf_many(hs3, gs)):
        assert torch.equal(m, api.psf(h, gg))


# P = Q M above one CTA: Q CTAs of a cluster per row / column (four-step split)
# P = 9000 (Q 8, M 1125), 8748 (Q 4, M 2187; two wavelengths: several slices per launch, loss
# partials of every CTA of every slice)
@pytest.mark.parametrize("N,pad,lams", [(4500, 2, [550e-9]), (4374, 2, [500e-9, 620e-9])])
def test_split_mixed_radix_psf_and_grad_vs_oracle(N, pad, lams):
    dx, z = 1e-6, 5e-3
    P = pad * N
    h = _h(N, 9950 + N)
    T = inputs.spot_target(P, N, len(lams), 9960 + N)
    g = Geometry.make(N, dx, z, lams, pad=pad)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    assert rel_l2(I, oracle.psf(h, dx, z, lams, pad=pad)) < TOL_PSF
    del I
    gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad(h, dx, z, lams, T, pad=pad)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref
    # the gradient from the fields a PSF call left in a gradient-sized workspace is the same
    ws = api.workspace(api.workspace_bytes(g, 3))
    api.psf(ht, g, ws=ws)
    g2, l2 = api.grad(ht, g, torch.from_numpy(T).cuda(), recompute=False, ws=ws)
    assert torch.equal(g2, gr) and torch.equal(l2, loss)


@pytest.mark.parametrize("N,pad,kw", [(6750, 2, {}), (13122, 1, dict(theta_x=0.02, src_d=-0.3))])
def test_split_mixed_radix_rows_vs_oracle(N, pad, kw):
    # P = 13500 (Q 5, M 2700), 13122 (pad 1, Q 3, M 4374; tilted converging illumination):
    # sampled PSF rows and the row-subset gradient against the oracle
    dx, z, lam = 1e-6, 20e-3, 550e-9
    P = pad * N
    h = _h(N, 9970 + N)
    e = oracle.incident(N, dx, lam, kw.get("theta_x", 0.0), 0.0, kw.get("src_d", 0.0)) if kw else None
    g = Geometry.make(N, dx, z, [lam], pad=pad, **kw)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g)
    rows = np.array([0, P // 3, P // 2 - 1, P // 2, P // 2 + 7, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    del I
    assert rel_l2(Ig, oracle.psf_rows(h, dx, z, lam, rows, pad=pad, e_in=e)) < TOL_PSF
    r = np.random.default_rng(9980 + N)
    grows = np.unique(np.concatenate([[P // 2], r.integers(0, P, 5)]))
    g_rows = r.standard_normal((grows.size, P)).astype(np.float32)
    G = torch.zeros((1, P, P), dtype=torch.float32, device="cuda")
    G[0, torch.from_numpy(grows).cuda()] = torch.from_numpy(g_rows).cuda()
    gr, _ = api.grad(ht, g, G, mode="vjp")
    drows = np.unique(np.concatenate([[0, N // 2, N - 1], r.integers(0, N, 3)]))
    got = gr[torch.from_numpy(drows).cuda()].cpu().numpy()
    del G, gr
    torch.cuda.empty_cache()
    ref = oracle.grad_rows(h, dx, z, lam, grows, g_rows, drows, pad=pad, e_in=e)
    assert rel_l2(got, ref) < TOL_GRAD


def test_table2_grid_28800_rows_vs_oracle():
    # Table 2's CHD / beam-shaping grid: a 3.6 mm DOE simulated at 0.25 um (14400^2, the 1800^2
    # design at 2 um upsampled 8x), padded to 28800 x 28800 (8 CTAs of 3600 points per
    # transform), 520.6 nm, 10 mm: sampled PSF rows and energy against the oracle
    N, f, dx, z, lam = 14400, 8, 0.25e-6, 10e-3, 520.6e-9
    P = 2 * N
    hl = _h(N // f, 9990)
    g = Geometry.make(N, dx, z, [lam], upsample=f)
    I = api.psf(torch.from_numpy(hl).cuda(), g)
    tot = I.double().sum().item()
    rows = np.array([0, P // 4, P // 2 - 1, P // 2, P // 2 + 1, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    del I
    torch.cuda.empty_cache()
    ref = oracle.psf_rows(oracle.upsample_nearest(hl, f), dx, z, lam, rows)
    assert rel_l2(Ig, ref) < TOL_PSF
    assert 0.5 * N * N < tot <= N * N * (1 + 1e-5)  # Parseval over the band


# prime factor 67 (Table 2's large-area grid 128640 x 85760 = 2^7 3 5 67 x 2^8 5 67): a
# direct-DFT stage inside the mixed-radix plan
@pytest.mark.parametrize("N,pad", [(670, 2), (1340, 1)])  # P = 1340 = 2^2 5 67
def test_prime_67_psf_and_grad_vs_oracle(N, pad):
    dx, z = 1e-6, 3e-3
    lams = [500e-9, 650e-9]
    P = pad * N
    h = _h(N, 9400 + N)
    T = inputs.spot_target(P, N, 2, 9410 + N)
    g = Geometry.make(N, dx, z, lams, pad=pad)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    assert rel_l2(I, oracle.psf(h, dx, z, lams, pad=pad)) < TOL_PSF
    gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad(h, dx, z, lams, T, pad=pad)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref


def test_prime_67_split_rows_vs_oracle():
    # P = 16080 = 8 x 2010 (2010 = 2 3 5 67): cluster split with a radix-67 stage per chunk
    N, dx, z, lam = 8040, 1e-6, 20e-3, 550e-9
    P = 2 * N
    h = _h(N, 9420)
    g = Geometry.make(N, dx, z, [lam])
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g)
    rows = np.array([0, P // 3, P // 2 - 1, P // 2, P - 1])
    Ig = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    del I
    assert rel_l2(Ig, oracle.psf_rows(h, dx, z, lam, rows)) < TOL_PSF
    r = np.random.default_rng(9421)
    grows = np.unique(np.concatenate([[P // 2], r.integers(0, P, 4)]))
    g_rows = r.standard_normal((grows.size, P)).astype(np.float32)
    G = torch.zeros((1, P, P), dtype=torch.float32, device="cuda")
    G[0, torch.from_numpy(grows).cuda()] = torch.from_numpy(g_rows).cuda()
    gr, _ = api.grad(ht, g, G, mode="vjp")
    drows = np.array([0, N // 2, N - 1])
    got = gr[torch.from_numpy(drows).cuda()].cpu().numpy()
    del G, gr
    torch.cuda.empty_cache()
    assert rel_l2(got, oracle.grad_rows(h, dx, z, lam, grows, g_rows, drows)) < TOL_GRAD


def test_split_mixed_radix_propagate_and_batching():
    # complex destination field on a split grid (P = 8748: Q 4 x 2187) against the oracle, and
    # two requests of that grid in one batched launch equal to their separate calls
    N, dx, z, lam = 4374, 1e-6, 5e-3, 550e-9
    h = _h(N, 9990 + 1)
    g = Geometry.make(N, dx, z, [lam])
    ht = torch.from_numpy(h).cuda()
    E = api.propagate(ht, g).cpu().numpy()[0]
    assert rel_l2(E, oracle.propagate(h, dx, z, lam)) < TOL_PSF
    del E
    h2 = torch.from_numpy(_h(N, 9990 + 2)).cuda()
    g2 = Geometry.make(N, dx, 8e-3, [480e-9, 640e-9], theta_x=0.01)
    many = api.psf_many([ht, h2], [g, g2])
    assert torch.equal(many[0], api.psf(ht, g))
    assert torch.equal(many[1], api.psf(h2, g2))


# -------------------------------------------------------------- circular band limit
def test_circular_band_mask_bit_exact():
    # the disc kt^2 + lt^2 < ceil((f_lim / du)^2): integer logic, equal to the oracle's mask
    for N, dx, z, lams in [(32, 0.25e-6, 5e-6, [400e-9, 700e-9]), (256, 2e-6, 20e-3, [550e-9]),
                           (180, 1e-6, 2e-3, [500e-9]), (16384, 1e-6, 50e-3, [550e-9])]:
        g = Geometry.make(N, dx, z, lams, bandlimit="circular")
        for j, lam in enumerate(lams):
            m = api.debug_band_mask(g, j).cpu().numpy()
            ref = oracle.band_mask(2 * N, dx, z, lam, bandlimit="circular")
            assert np.array_equal(m, ref), (N, j)


@pytest.mark.parametrize("N,pad", [(256, 2), (180, 2), (128, 1)])
def test_circular_band_psf_and_grad_vs_oracle(N, pad):
    dx, z = 2e-6, 20e-3 * N / 256
    lams = [450e-9, 550e-9, 650e-9]
    P = pad * N
    h = _h(N, 1301)
    T = inputs.spot_target(P, N, 3, 2301)
    g = Geometry.make(N, dx, z, lams, pad=pad, bandlimit="circular")
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    ref = oracle.psf(h, dx, z, lams, pad=pad, bandlimit="circular")
    assert rel_l2(I, ref) < TOL_PSF, rel_l2(I, ref)
    gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda())
    rg, rloss = oracle.grad(h, dx, z, lams, T, pad=pad, bandlimit="circular")
    assert rel_l2(gr.cpu().numpy(), rg) < TOL_GRAD
    assert abs(loss.item() - rloss) <= 1e-5 * rloss
    # the disc removes energy the square band keeps
    assert I.sum() < api.psf(ht, Geometry.make(N, dx, z, lams, pad=pad)).cpu().numpy().sum()


def test_circular_band_split_grid_rows_vs_oracle():
    # 16384^2 DOE on the 32768^2 split grid at 50 mm: the square band is inactive there
    # (kmax = P / 2) while the disc still cuts the corners of the spectrum
    N, dx, z, lam = 16384, 1e-6, 50e-3, 550e-9
    P = 2 * N
    assert oracle.kmax(lam, dx, P, z) == P // 2
    assert oracle.m_lim(lam, dx, P, z, "circular") < 2 * (P // 2) ** 2
    h = _h(N, 1305)
    g = Geometry.make(N, dx, z, [lam], bandlimit="circular")
    I = api.psf(torch.from_numpy(h).cuda(), g)
    rows = np.array([0, P // 4, P // 2, P // 2 + 5, P - 1])
    got = I[0, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    ref = oracle.psf_rows(h, dx, z, lam, rows, bandlimit="circular")
    assert rel_l2(got, ref) < TOL_PSF, rel_l2(got, ref)


# -------------------------------------------------------------- degenerate bands
@pytest.mark.parametrize("N,dx,z,lams,regime", [
    (128, 1e-6, 0.1, [550e-9], "kmax0"),            # only the zero-frequency row and column pass
    (128, 1e-6, 0.05, [550e-9], "kmax1"),
    (90, 1e-6, 0.1, [550e-9], "kmax0"),             # mixed radix, P = 180
    (64, 0.25e-6, 5e-6, [400e-9, 700e-9], "evanescent"),  # pitch below lambda / 2: the evanescent cut binds
])
def test_degenerate_bands_vs_oracle(N, dx, z, lams, regime):
    P = 2 * N
    for lam in lams:
        k = oracle.kmax(lam, dx, P, z)
        if regime == "kmax0":
            assert k == 0
        elif regime == "kmax1":
            assert k == 1
        else:  # the evanescent disc cuts the corners of the square band
            assert oracle.m_ev(lam, dx, P) <= 2 * k * k
    h = _h(N, 9300 + N)
    T = inputs.spot_target(P, N, len(lams), 9400 + N)
    g = Geometry.make(N, dx, z, lams)
    ht = torch.from_numpy(h).cuda()
    I = api.psf(ht, g).cpu().numpy()
    assert np.isfinite(I).all()
    assert rel_l2(I, oracle.psf(h, dx, z, lams)) < TOL_PSF, rel_l2(I, oracle.psf(h, dx, z, lams))
    gr, loss = api.grad(ht, g, torch.from_numpy(T).cuda())
    gref, lref = oracle.grad(h, dx, z, lams, T)
    assert rel_l2(gr.cpu().numpy(), gref) < TOL_GRAD
    assert abs(loss.item() - lref) <= 1e-5 * lref
