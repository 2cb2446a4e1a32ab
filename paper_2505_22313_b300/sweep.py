"""Per-configuration timing of the library's passes (PSF and gradient).

    python -m paper_2505_22313_b300.sweep [--configs small,rgb,gradient,large_area,wiener,design_table2_3600] [--reps K]

Each configuration runs the PSF (and, where listed, the L2 gradient against the spot-array
target with recomputed fields) K times after warm-up, timed with CUDA events on the current
stream, and prints one JSON line: wall time per call, field-samples/s, and the median device
time of every traced pass.  Inputs are the seeded synthetic heights and targets of
``inputs``; nothing here checks results (the tests do).
"""
from __future__ import annotations

import argparse
import json

CONFIGS = {
    # name: (N, pitch m, z m, wavelengths m, gradient?[, nearest-upsampling factor of the heights
    #        [, parametric incident field]])
    "small": (256, 2e-6, 20e-3, [550e-9], True),
    "rgb": (4096, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9], True),
    "gradient": (8192, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9], True),
    "grid_16384": (8192, 1e-6, 50e-3, [550e-9], False),  # one wavelength: ~3.3 GB on the device
    "grid_32768": (16384, 1e-6, 50e-3, [550e-9], True),
    "large_area": (32768, 1e-6, 100e-3, [550e-9], True),
    # the RGB geometry designed on a 1024^2 layout at 4 um, nearest-upsampled 4x in pass A
    "rgb_layout4": (4096, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9], True, 4),
    # the same layout interpolated with Lanczos-3 instead (a pre-pass and its transpose)
    "rgb_layout4_lanczos": (4096, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9], True, 4, dict(lanczos=True)),
    # Table 2's 3600 x 3600 grid: a 3.6 mm DOE at 2 um, 520.6 nm, hologram plane at 10 mm
    # (mixed-radix transforms)
    "table2_3600": (1800, 2e-6, 10e-3, [520.6e-9], True),
    # a split mixed-radix grid small enough to profile: 4500^2 DOE padded to 9000 x 9000
    # (clusters of 8 CTAs of 1125 points)
    "split_9000": (4500, 1e-6, 5e-3, [550e-9], False),
    # Table 2's CHD / beam-shaping grid: the 1800^2 design at 2 um upsampled 8x onto 14400^2 at
    # 0.25 um, padded to 28800 x 28800 (clusters of 8 CTAs of 3600 points)
    "table2_28800": (14400, 0.25e-6, 10e-3, [520.6e-9], True, 8),
    # Table 2's broadband-imaging grid: a 10 mm DOE at 0.5 um (20000^2) padded to 40000 x 40000,
    # six wavelengths over 400-700 nm (clusters of 8 CTAs of 5000 points); ~200 GB for the gradient
    "table2_40000x6": (20000, 0.5e-6, 50e-3, [400e-9, 460e-9, 520e-9, 580e-9, 640e-9, 700e-9], True),
    # the RGB geometry lit by a tilted wave converging to 200 mm (evaluated in the DOE-row passes)
    "rgb_tilted_converging": (4096, 1e-6, 50e-3, [450e-9, 550e-9, 650e-9], True, 1,
                              dict(theta_x=0.01, theta_y=-0.005, src_d=-0.2)),
}


def run(name: str, reps: int, grad: bool = True) -> dict:
    import torch

    from . import _lib, api, inputs
    from .api import Geometry

    N, dx, z, lams, do_grad, *rest = CONFIGS[name]
    f = rest[0] if rest else 1
    illum = rest[1] if len(rest) > 1 else {}
    do_grad = do_grad and grad
    P = 2 * N
    g = Geometry.make(N, dx, z, lams, upsample=f, **illum)
    h = inputs.heights_device(N // f, 1000 + N, "cuda")
    ws = api.workspace(api.workspace_bytes(g, _lib.DOE_OP_GRAD if do_grad else _lib.DOE_OP_PSF))
    out = torch.empty((g.L, P, P), device="cuda")
    for _ in range(2):
        api.psf(h, g, out=out, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    api.trace_enable(reps * 8 + 64)
    e0.record()
    for _ in range(reps):
        api.psf(h, g, out=out, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    psf_ms = e0.elapsed_time(e1) / reps
    row = {"config": name, "N": N, "P": P, "wavelengths": g.L, "upsample": f, "illum": illum, "psf_ms": round(psf_ms, 3),
           "field_samples_per_s": g.L * P * P / (psf_ms / 1e3)}
    recs = api.trace_read()
    del out
    if do_grad:
        T = torch.from_numpy(inputs.spot_target(P, N, g.L, 2000 + N)).cuda()
        api.grad(h, g, T, ws=ws)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            api.grad(h, g, T, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        row["grad_ms"] = round(e0.elapsed_time(e1) / reps, 3)
        recs += api.trace_read()
        del T
    api.trace_enable(0)
    per: dict[str, list[float]] = {}
    for n, ms in recs:
        per.setdefault(n, []).append(ms)
    row["passes_ms"] = {k: round(sorted(v)[len(v) // 2], 3) for k, v in per.items()}
    del ws, h
    torch.cuda.empty_cache()
    return row


def run_wiener(reps: int, C: int = 3, H: int = 2048, W: int = 2048, P: int = 8192) -> dict:
    """Wiener deconvolution (Eq. 9) of C seeded H x W images with seeded P x P PSFs."""
    import numpy as np
    import torch

    from . import _lib, api, inputs

    rng = np.random.default_rng(2048)
    psf = torch.from_numpy(rng.random((C, P, P), dtype=np.float32) ** 4).cuda()
    y = torch.from_numpy(inputs.image(C, H, W, 2002)).cuda()
    out = torch.empty_like(y)
    ws = api.workspace(int(_lib.load().doe_wiener_workspace_bytes(C, H, W)))
    for _ in range(3):
        out = api.wiener(psf, y, 5e-4, out=out, ws=ws)
    torch.cuda.synchronize()
    api.trace_enable(reps * 4 + 16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        api.wiener(psf, y, 5e-4, out=out, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    recs = api.trace_read()
    api.trace_enable(0)
    per: dict[str, list[float]] = {}
    for n, ms in recs:
        per.setdefault(n, []).append(ms)
    ms = e0.elapsed_time(e1) / reps
    return {"config": f"wiener_{C}x{H}x{W}", "wiener_ms": round(ms, 4), "pixels_per_s": C * H * W / (ms / 1e3),
            "passes_ms": {k: round(sorted(v)[len(v) // 2], 4) for k, v in per.items()}}


def run_design(reps: int, name: str = "gradient") -> dict:
    """Design-loop iterations (doe_grad + doe_adam_step) per second on a gradient workload."""
    import torch

    from . import api, design, inputs
    from .api import Geometry

    N, dx, z, lams, _, *rest = CONFIGS[name]
    f = rest[0] if rest else 1
    illum = rest[1] if len(rest) > 1 else {}
    P = 2 * N
    g = Geometry.make(N, dx, z, lams, upsample=f, **illum)
    h0 = inputs.heights_device(N // f, 1000 + N, "cuda")
    T = torch.from_numpy(inputs.spot_target(P, N, g.L, 2000 + N)).cuda()
    design.optimize(h0, g, T, 2)
    torch.cuda.synchronize()
    api.trace_enable(reps * 16 + 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, losses = design.optimize(h0, g, T, reps)
    e1.record()
    torch.cuda.synchronize()
    recs = api.trace_read()
    api.trace_enable(0)
    adam = [ms for n, ms in recs if n == "adam_step"]
    ms = e0.elapsed_time(e1) / reps
    return {"config": f"design_{name}", "iteration_ms": round(ms, 3), "iterations_per_s": round(1e3 / ms, 2),
            "adam_step_ms": round(sorted(adam)[len(adam) // 2], 4) if adam else None,
            "loss_first_last": [float(losses[0]), float(losses[-1])]}


def run_design_radial(reps: int, name: str = "rgb") -> dict:
    """Radially symmetric design iterations (doe_radial_heights, doe_grad, doe_radial_grad, Adam
    on 9 coefficients) per second on a configuration."""
    import torch

    from . import api, design, inputs
    from .api import Geometry

    N, dx, z, lams, *_ = CONFIGS[name]
    P = 2 * N
    g = Geometry.make(N, dx, z, lams)
    c0 = torch.zeros(9, device="cuda")
    c0[0], c0[1] = 0.6e-6, -0.3e-6
    T = torch.from_numpy(inputs.spot_target(P, N, g.L, 2000 + N, grid=1)).cuda()
    design.optimize_radial(c0, g, T, 2, 3e-9)
    torch.cuda.synchronize()
    api.trace_enable(reps * 16 + 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, losses = design.optimize_radial(c0, g, T, reps, 3e-9)
    e1.record()
    torch.cuda.synchronize()
    recs = api.trace_read()
    api.trace_enable(0)
    per: dict[str, list[float]] = {}
    for n, ms in recs:
        per.setdefault(n, []).append(ms)
    ms = e0.elapsed_time(e1) / reps
    return {"config": f"design_radial_{name}", "iteration_ms": round(ms, 3),
            "passes_ms": {k: round(sorted(v)[len(v) // 2], 4) for k, v in per.items()},
            "loss_first_last": [float(losses[0]), float(losses[-1])]}


def main():
    from . import api

    ap = argparse.ArgumentParser(description="per-configuration pass timing")
    ap.add_argument("--configs", default=",".join(CONFIGS))
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-grad", action="store_true", help="time the PSF only")
    args = ap.parse_args()
    api.init()
    for name in args.configs.split(","):
        name = name.strip()
        if name == "wiener":
            row = run_wiener(args.reps)
        elif name.startswith("radial"):
            # "radial" times the radially symmetric design loop on the RGB geometry; "radial_<config>"
            row = run_design_radial(args.reps, name[len("radial_"):] if name.startswith("radial_") else "rgb")
        elif name.startswith("design"):
            # "design" times the gradient workload; "design_<config>" any configuration
            row = run_design(args.reps, name[len("design_"):] if name.startswith("design_") else "gradient")
        else:
            row = run(name, args.reps, grad=not args.no_grad)
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
