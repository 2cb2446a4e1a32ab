"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the diffraction method (no phase, no transform, no
propagation): it only draws and shapes random inputs.  The tests feed the very same
arrays to the CUDA library and to the FP64 oracle; the benchmark uses them as its
synthetic workload.  Nothing here depends on the CUDA library or on the oracle.

Recipes (seeds: heights 1000 + c, images and targets 2000 + c, request stream 3000):
  heights  raw ~ U[0, 1) float32 (PCG64, numpy default_rng(seed)); separable Gaussian
           smoothing, sigma = 2 px, radius 8 (weights normalised), periodic boundary,
           evaluated in FP64; rounded to float32; affine rescale of that float32 field so
           that its minimum is 0 and its maximum is hmax = 1.2 um exactly; float32 metres.
           (Sec. 3.2's contrast-curve footnote ties ~1.2 um of resist to a 2 pi phase at
           550 nm, which is why the heights span [0, 1.2] um.)
  image    C x H x W float32: iid U[0, 1), then 64 filled disks painted over it, each with
           radius U[8, 128] px, a uniform random centre, and one U[0, 1) value per channel.
  target   8 x 8 lattice of Gaussian spots per wavelength (the beam-splitter task of
           Sec. 5.3): pitch P/32, sigma 8 px, each centre jittered by U[-P/256, P/256] in
           both axes, lattice centred at (P/2, P/2), scaled so that each wavelength's
           target sums to N^2 (the energy of a unit-amplitude N x N aperture).
  flat-top 8 x 8 regular lattice of equal-intensity discs (Sec. 5.3's flat-top spot array),
           pitch P/32, radius pitch/4, centred at (P/2, P/2), summing to N^2.
  requests Poisson arrivals at a given rate; side N uniform in {1024, ..., 16384};
           1..31 wavelengths uniform in [400, 700] nm; z uniform in [10, 100] mm;
           pitch 1 um; per-request heights seed 100000 + request id.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HMAX = 1.2e-6


def _gauss_weights(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    return w / w.sum()


def _smooth_rows_periodic(block: np.ndarray, w: np.ndarray) -> np.ndarray:
    from scipy.ndimage import correlate1d

    return correlate1d(block, w, axis=1, mode="wrap")


def heights(N: int, seed: int, hmax: float = HMAX, sigma: float = 2.0, radius: int = 8) -> np.ndarray:
    """Smoothed random DOE height map, float32 metres, [N][N]."""
    rng = np.random.default_rng(seed)
    raw = rng.random((N, N), dtype=np.float32)
    w = _gauss_weights(sigma, radius)
    out = np.empty((N, N), np.float32)
    B = min(N, 256)
    for r0 in range(0, N, B):
        b = min(B, N - r0)  # the last block is shorter when B does not divide N
        idx = np.arange(r0 - radius, r0 + b + radius) % N
        blk = _smooth_rows_periodic(raw[idx].astype(np.float64), w)
        from scipy.ndimage import correlate1d

        acc = correlate1d(blk, w, axis=0, mode="constant")[radius:radius + b]
        out[r0:r0 + b] = acc.astype(np.float32)
    mn = float(out.min())
    mx = float(out.max())
    scale = hmax / (mx - mn)
    for r0 in range(0, N, B):
        out[r0:r0 + B] = ((out[r0:r0 + B].astype(np.float64) - mn) * scale).astype(np.float32)
    return out


def heights_device(N: int, seed: int, device, hmax: float = HMAX, sigma: float = 2.0, radius: int = 8):
    """Seeded smoothed heights generated on a CUDA device (the serving workload's requests):
    torch's device RNG U[0, 1), the same separable periodic Gaussian smoothing and affine
    rescale to [0, hmax] as heights(), in float32.  Deterministic for a given seed and device
    type; not bit-identical to heights() (different random generator)."""
    import torch
    import torch.nn.functional as F

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.rand((N, N), generator=g, device=device, dtype=torch.float32)
    w = torch.tensor(_gauss_weights(sigma, radius), dtype=torch.float32, device=device).view(1, 1, -1)
    # periodic correlation along x (rows as a batch), then along y: out[j] = sum_i w[i] x[j + i - radius]
    x = F.conv1d(F.pad(x.view(N, 1, N), (radius, radius), mode="circular"), w).view(N, N)
    x = F.conv1d(F.pad(x.t().contiguous().view(N, 1, N), (radius, radius), mode="circular"), w).view(N, N).t()
    mn, mx = x.min(), x.max()
    return ((x - mn) * (hmax / (mx - mn))).contiguous()


def image(C: int, H: int, W: int, seed: int, n_disks: int = 64) -> np.ndarray:
    """C x H x W float32 test scene: iid uniform noise with filled disks painted on top."""
    rng = np.random.default_rng(seed)
    img = rng.random((C, H, W), dtype=np.float32)
    yy = np.arange(H)[:, None]
    xx = np.arange(W)[None, :]
    for _ in range(n_disks):
        r = rng.uniform(8, 128)
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        vals = rng.random(C).astype(np.float32)
        y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
        m = (yy[y0:y1] - cy) ** 2 + (xx[:, x0:x1] - cx) ** 2 <= r * r
        for c in range(C):
            img[c, y0:y1, x0:x1][m] = vals[c]
    return img


def _spot_tiles(P: int, N: int, n_lambda: int, seed: int, grid: int = 8, sigma: float = 8.0):
    """The non-zero tiles of spot_target: (wavelength, y0, x0, float32 tile) in drawing order."""
    rng = np.random.default_rng(seed)
    pitch = P / 32.0
    jit = P / 256.0
    rad = int(np.ceil(5 * sigma))
    offs = (np.arange(grid) - (grid - 1) / 2.0) * pitch + P / 2.0
    out = []
    for j in range(n_lambda):
        spots = []
        for cy0 in offs:
            for cx0 in offs:
                cy = cy0 + rng.uniform(-jit, jit)
                cx = cx0 + rng.uniform(-jit, jit)
                spots.append((cy, cx))
        total = 0.0
        tiles = []
        for cy, cx in spots:
            y0, y1 = max(0, int(cy) - rad), min(P, int(cy) + rad + 1)
            x0, x1 = max(0, int(cx) - rad), min(P, int(cx) + rad + 1)
            ys = np.arange(y0, y1)[:, None]
            xs = np.arange(x0, x1)[None, :]
            g = np.exp(-((ys - cy) ** 2 + (xs - cx) ** 2) / (2 * sigma * sigma))
            tiles.append((y0, x0, g))
            total += g.sum()
        scale = float(N) * float(N) / total
        out += [(j, y0, x0, (g * scale).astype(np.float32)) for y0, x0, g in tiles]
    return out


def spot_target(P: int, N: int, n_lambda: int, seed: int, grid: int = 8, sigma: float = 8.0) -> np.ndarray:
    """[L][P][P] float32 Gaussian spot-array targets, each summing to N^2."""
    T = np.zeros((n_lambda, P, P), np.float32)
    for j, y0, x0, g in _spot_tiles(P, N, n_lambda, seed, grid, sigma):
        T[j, y0:y0 + g.shape[0], x0:x0 + g.shape[1]] += g
    return T


def spot_target_device(P: int, N: int, n_lambda: int, seed: int, device, grid: int = 8, sigma: float = 8.0):
    """spot_target assembled directly in device memory (the same values; for grids whose
    target is too large to stage on the host)."""
    import torch

    T = torch.zeros((n_lambda, P, P), dtype=torch.float32, device=device)
    for j, y0, x0, g in _spot_tiles(P, N, n_lambda, seed, grid, sigma):
        T[j, y0:y0 + g.shape[0], x0:x0 + g.shape[1]] += torch.from_numpy(g).to(device)
    return T


def flat_top_target(P: int, N: int, n_lambda: int, grid: int = 8, pitch: float | None = None,
                    radius: float | None = None) -> np.ndarray:
    """[L][P][P] float32 beam-splitter targets: a regular grid x grid lattice of flat-top,
    equal-intensity discs (pitch P/32 and radius pitch/4 by default) centred at (P/2, P/2),
    each wavelength's target summing to N^2."""
    pitch = P / 32.0 if pitch is None else float(pitch)
    radius = pitch / 4.0 if radius is None else float(radius)
    offs = (np.arange(grid) - (grid - 1) / 2.0) * pitch + P / 2.0
    ys = np.arange(P, dtype=np.float64)[:, None]
    xs = np.arange(P, dtype=np.float64)[None, :]
    m = np.zeros((P, P), bool)
    for cy in offs:
        for cx in offs:
            y0, y1 = max(0, int(cy - radius) - 1), min(P, int(cy + radius) + 2)
            x0, x1 = max(0, int(cx - radius) - 1), min(P, int(cx + radius) + 2)
            m[y0:y1, x0:x1] |= (ys[y0:y1] - cy) ** 2 + (xs[:, x0:x1] - cx) ** 2 <= radius * radius
    T = np.where(m, float(N) * float(N) / m.sum(), 0.0).astype(np.float32)
    return np.broadcast_to(T, (n_lambda, P, P)).copy()


def gaussian_beam(N: int, dx: float, w0: float) -> np.ndarray:
    """Unit-peak Gaussian amplitude exp(-r^2 / w0^2) sampled on the N x N DOE grid, with
    the beam axis at DOE sample (N/2, N/2) (the optical axis of a 2x padded grid)."""
    c = (np.arange(N) - N // 2) * dx
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    return np.exp(-r2 / (w0 * w0)).astype(np.complex128)


@dataclass
class Request:
    rid: int
    arrival_s: float
    N: int
    lambdas: np.ndarray
    z: float
    dx: float = 1e-6
    seed: int = 0
    n_index: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def P(self) -> int:
        return 2 * self.N


def request_stream(n: int, rate_hz: float, seed: int = 3000,
                   sides=(1024, 2048, 4096, 8192, 16384), max_lambda: int = 31) -> list[Request]:
    """Seeded Poisson request trace for the serving workload."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate_hz)
        N = int(rng.choice(sides))
        L = int(rng.integers(1, max_lambda + 1))
        lams = rng.uniform(400e-9, 700e-9, size=L)
        z = float(rng.uniform(10e-3, 100e-3))
        out.append(Request(rid=rid, arrival_s=t, N=N, lambdas=lams, z=z, dx=1e-6,
                           seed=100000 + rid, n_index=np.full(L, 1.46)))
    return out
