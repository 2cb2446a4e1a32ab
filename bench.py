#!/usr/bin/env python3
"""Benchmark of the DOE scalar-diffraction path on B300.

Headline workload (RGB design evaluation, the default): a 4096 x 4096 DOE at 1 um pitch,
heights in [0, 1.2] um (seeded, smoothed), wavelengths 450/550/650 nm, n = 1.46, z = 50 mm,
padded to 8192 x 8192: three PSFs, then the FFT convolution of a seeded 3 x 2048 x 2048 image
with them.  One step is that whole chain.  Metric: field-samples/s = (wavelengths x P^2) per
step / step time.

The default line also carries a "configs" block with one sub-record per other workload, each
timed the same way (CUDA events on the launching stream, per-pass device times, the dominant
pass's roofline, clocks, error against the FP64 oracle):
  1  plain_small_256     256^2 DOE, 512^2 grid, 550 nm, PSF (latency; L2 flushed between steps)
  3  gradient_8192       8192^2 DOE, 16384^2 grid, 3 wavelengths, PSF + L2 gradient (recomputed fields)
  4  large_area_32768    32768^2 DOE, 65536^2 grid, 550 nm, z = 100 mm, PSF + L2 gradient (recomputed)
  5  serving_poisson_mix a seeded Poisson trace of DOE requests, continuous batching vs one at a time

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 1..5]

--config N makes workload N the main line (no sub-records).  N > 1 GPUs run under torchrun
as independent replicas (one per GPU, weak scaling: the path has no exchange step between
GPUs).  The reference arm is the FP64 CPU oracle.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "DOE PSF field-samples/s & % HBM roofline at stated FP64 error; p50/p99 latency"
UNIT = "field-samples/s"

CONFIGS = {
    1: dict(workload="plain_small_256", N=256, dx=2e-6, z=20e-3, lambdas=[550e-9], step="psf", h_seed=1001),
    2: dict(workload="rgb_design_eval_4096", N=4096, dx=1e-6, z=50e-3, lambdas=[450e-9, 550e-9, 650e-9],
            step="psf+render", C=3, H=2048, W=2048, h_seed=1002, img_seed=2002),
    3: dict(workload="gradient_8192", N=8192, dx=1e-6, z=50e-3, lambdas=[450e-9, 550e-9, 650e-9], step="psf+grad",
            h_seed=1003, tgt_seed=2003),
    4: dict(workload="large_area_32768", N=32768, dx=1e-6, z=100e-3, lambdas=[550e-9], step="psf+grad",
            h_seed=1004, tgt_seed=2004),
    # Table 2's grids (non-power-of-two sides, mixed-radix passes): a 3.6 mm DOE at 2 um, 520.6 nm,
    # hologram plane at 10 mm (3600^2 grid); the 1800^2 design upsampled 8x (nearest) onto 14400^2
    # at 0.25 um (28800^2 grid); and a 4500^2 DOE padded to 9000^2 (clusters of 8 CTAs of 1125 points)
    "table2_3600": dict(workload="table2_3600", N=1800, dx=2e-6, z=10e-3, lambdas=[520.6e-9], step="psf+grad",
                        h_seed=2800, tgt_seed=3800),
    "table2_28800": dict(workload="table2_28800", N=14400, dx=0.25e-6, z=10e-3, lambdas=[520.6e-9],
                         step="psf+grad", upsample=8, h_seed=15400, tgt_seed=16400),
    "split_9000": dict(workload="split_9000", N=4500, dx=1e-6, z=5e-3, lambdas=[550e-9], step="psf", h_seed=5500),
    # the serving mix's largest requests: a 16384^2 DOE padded to 32768^2 (columns and rows split
    # over clusters of 4 CTAs of 8192 points), PSF + L2 gradient
    "grid_32768": dict(workload="grid_32768", N=16384, dx=1e-6, z=50e-3, lambdas=[550e-9], step="psf+grad",
                       h_seed=6384, tgt_seed=7384),
}
SERVING = dict(workload="serving_poisson_mix", requests=40, rate_hz=200.0, seed=3000,
               sides=(1024, 2048, 4096, 8192, 16384), max_lambda=31)
N_INDEX = 1.46
PAD = 2
WL = CONFIGS[2]
SUBS = ((1, 50), (3, 20), (4, 5), ("table2_3600", 20))  # sub-records of the default line: (config, timed steps)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _config(cfg, extra=None):
    P = PAD * cfg["N"]
    c = {"workload": cfg["workload"], "doe": f"{cfg['N']}x{cfg['N']}", "pitch_um": cfg["dx"] * 1e6,
         "grid": f"{P}x{P}", "lambdas_nm": [round(l * 1e9, 1) for l in cfg["lambdas"]], "z_mm": cfg["z"] * 1e3,
         "step": cfg["step"]}
    if "C" in cfg:
        c["render"] = f"{cfg['C']}x{cfg['H']}x{cfg['W']}"
    c["l2_flush"] = ("256 MB buffer written between timed steps" if P * P * 8 * len(cfg["lambdas"]) < (256 << 20)
                     else f"inputs larger than L2 ({_step_bytes(cfg) / 1e9:.1f} GB moved per step)")
    if extra:
        c.update(extra)
    return c


def _step_bytes(cfg):
    P, S = PAD * cfg["N"], len(cfg["lambdas"])
    return 3 * 8 * S * P * P  # order of magnitude of one step's traffic (three passes over one field per slice)


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def _band_w(kmax: int, P: int) -> int:
    """Stored columns of one slice: the band-compacted segments for power-of-two P <= 16384
    with the band limit active, else all P columns (split grids are stored in sub-transform
    order, mixed-radix grids in natural order)."""
    if kmax >= P // 2 or P > 16384 or P & (P - 1):
        return P
    return ((kmax + 2) & ~1) + ((kmax + 1) & ~1)


def _algorithmic_bytes(kmax, P, N, C=0, H=0, W=0, NL=None):
    """Compulsory DRAM bytes of one launch of each pass (band-pruned storage; the fields of
    the gradient's recomputed forward passes count like the forward ones).  NL: side of the
    height layout (N / upsampling factor)."""
    S = len(kmax)
    NL = N if NL is None else NL
    w = sum(_band_w(k, P) for k in kmax)
    tab = sum((k + 1) ** 2 for k in kmax) * 8
    qf = P // 8192 if P > 16384 else 1
    return {
        "transfer_table": tab,
        "pass_a_rows": S * NL * NL * 4 + N * w * 8,
        "pass_b_columns": N * w * 8 + P * w * 8 + tab,
        "pass_c_rows": P * w * 8 + S * P * P * 4,
        "pass_c_adjoint_rows": 2 * P * w * 8 + S * P * P * 4 + S * P * qf * 8,
        "pass_b_adjoint_columns": P * w * 8 + N * w * 8 + tab,
        "pass_a_adjoint_rows": N * w * 8 + S * NL * NL * 4 + N * N * 4,
        "loss_reduce": S * P * qf * 8,
        "render_rows": 2 * C * H * W * 4 + 2 * C * H * (W + 1) * 8,
        "render_columns": 3 * C * H * (W + 1) * 8,
        "render_output": C * H * (W + 1) * 8 + C * H * W * 4,
    }


def _algorithmic_flops(kmax, P, N, C=0, H=0, W=0):
    """FP32 flops of one launch of each pass, counting 5 n log2 n per length-n complex
    transform (the usual FFT convention) plus the pointwise products."""
    S = len(kmax)
    w = sum(_band_w(k, P) for k in kmax)
    f = 5 * P * int(math.log2(P))  # one length-P transform
    fr = 5 * 2 * W * int(math.log2(2 * W)) if W else 0
    fc = 5 * 2 * H * int(math.log2(2 * H)) if H else 0
    return {
        "transfer_table": 0,
        "pass_a_rows": S * N * f,
        "pass_b_columns": w * (2 * f + 6 * P),
        "pass_c_rows": S * P * (f + 3 * P),
        "pass_c_adjoint_rows": S * P * (2 * f + 12 * P),
        "pass_b_adjoint_columns": w * (2 * f + 6 * P),
        "pass_a_adjoint_rows": S * N * (f + 8 * N),
        "loss_reduce": 0,
        "render_rows": C * H * fr,
        "render_columns": C * (W + 1) * (3 * fc + 6 * 2 * H),
        "render_output": (C * H // 2) * fr,
    }


def _fp32_peak_tflops(dev, clk):
    """FP32 ALU peak from the device's SM count and the SM clock sampled during the timed
    region (NVML; the maximum clock if no sample was taken): SMs x 128 FP32 lanes x 2 flops."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    src = "sampled median SM clock" if clk.get("sm_mhz") else "maximum SM clock"
    if not mhz:
        mhz, src = 2032.0, "nominal maximum SM clock (no NVML sample)"
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({src})"


def _source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2505_22313_b300" / "csrc").glob("*")):
        if f.suffix in (".cu", ".cuh", ".h"):
            h.update(f.read_bytes())
    return h.hexdigest()[:16]


def _traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("source_sha") != _source_hash():
        return None
    e = d.get("workloads", {}).get(workload, {}).get(kernel)
    return e.get("dram_bytes_per_launch") if e else None


# kernel (demangled ncu name) -> pass name of the library's trace, for the PSF + render step
_TRAFFIC_KERNELS = (("htab_kernel", "transfer_table"), ("pass_a_kernel", "pass_a_rows"),
                    ("pass_b_kernel", "pass_b_columns"), ("pass_c_kernel", "pass_c_rows"),
                    ("render_rows_kernel", "render_rows"), ("render_cols_kernel", "render_columns"),
                    ("render_out_kernel", "render_output"))


def ingest_traffic(csv_path: str, workload: str, command: str) -> dict:
    """Writes profiles/traffic.json from an ncu CSV of dram__bytes_read.sum,
    dram__bytes_write.sum and gpu__time_duration.sum (one row per metric and launch): per pass
    of a PSF + render step, the mean DRAM bytes per launch, keyed on the current kernel sources.
    Entries of other workloads taken on the same sources are kept."""
    import csv
    import re

    launches = {}
    with open(csv_path, newline="") as f:
        rows = [r for r in csv.reader(line for line in f if line.startswith('"'))]
    head = rows[0]
    ix = {k: head.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Value")}
    for r in rows[1:]:
        e = launches.setdefault(r[ix["ID"]], {"kernel": r[ix["Kernel Name"]]})
        e[r[ix["Metric Name"]]] = float(r[ix["Metric Value"]].replace(",", ""))
    per = {}
    for e in launches.values():
        name = next((p for k, p in _TRAFFIC_KERNELS if re.search(rf"\b{k}\b", e["kernel"])), None)
        if name is None or "dram__bytes_read.sum" not in e:
            continue
        per.setdefault(name, []).append(e)
    out = {}
    for name, es in per.items():
        rd = sum(e["dram__bytes_read.sum"] for e in es) / len(es)
        wr = sum(e["dram__bytes_write.sum"] for e in es) / len(es)
        dur = sum(e.get("gpu__time_duration.sum", 0.0) for e in es) / len(es)
        out[name] = {"dram_bytes_per_launch": int(rd + wr), "read_bytes": int(rd), "write_bytes": int(wr),
                     "duration_ns": round(dur, 1), "launches": len(es), "kernel": es[0]["kernel"]}
    p = ROOT / "profiles" / "traffic.json"
    sha = _source_hash()
    d = json.loads(p.read_text()) if p.exists() else {}
    if d.get("source_sha") != sha:
        d = {}
    d.update({"_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch (mean over the captured launches) "
                       "from ncu captures of the named workloads; valid only for the kernel sources with this source_sha",
              "source_sha": sha})
    d.setdefault("workloads", {})[workload] = {"_command": command, **out}
    p.write_text(json.dumps(d, indent=1) + "\n")
    return d


class _Nvml:
    """Read-only NVML queries: pynvml when importable, else the driver's libnvidia-ml through
    ctypes (same public entry points)."""

    CLOCK_SM = 1  # NVML_CLOCK_SM

    def __init__(self):
        try:
            import pynvml as nv

            nv.nvmlInit()
            self.nv, self.lib = nv, None
        except ImportError:
            import ctypes

            self.nv, self.lib, self.ct = None, ctypes.CDLL("libnvidia-ml.so.1"), ctypes
            if self.lib.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")

    def handle(self, bus: str | None, index: int):
        if self.nv:
            try:
                return self.nv.nvmlDeviceGetHandleByPciBusId(bus) if bus else self.nv.nvmlDeviceGetHandleByIndex(index)
            except Exception:
                return self.nv.nvmlDeviceGetHandleByIndex(index)
        h = self.ct.c_void_p()
        if not bus or self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), self.ct.byref(h)) != 0:
            if self.lib.nvmlDeviceGetHandleByIndex_v2(self.ct.c_uint(index), self.ct.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        return h

    def _uint(self, fn, h, *args):
        v = self.ct.c_uint()
        if getattr(self.lib, fn)(h, *args, self.ct.byref(v)) != 0:
            raise RuntimeError(fn)
        return v.value

    def sm_clock(self, h):
        return self.nv.nvmlDeviceGetClockInfo(h, self.CLOCK_SM) if self.nv else self._uint("nvmlDeviceGetClockInfo", h, self.CLOCK_SM)

    def sm_max(self, h):
        return self.nv.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM) if self.nv else self._uint("nvmlDeviceGetMaxClockInfo", h, self.CLOCK_SM)

    def reasons(self, h):
        if self.nv:
            get = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
            return get(h)
        v = self.ct.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(h, self.ct.byref(v)) != 0:
            raise RuntimeError("clock event reasons")
        return v.value


class _Clocks:
    """SM clock and clock-event reasons of the device, sampled during the timed region through
    NVML (read-only queries): one sample on entry, one every 5 ms from a thread, one on exit, so
    that a region of a few tens of milliseconds still has several samples."""

    REASONS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
               ("hw_thermal_slowdown", 0x40))

    def __init__(self, dev: int):
        self.dev = dev
        self.h = None
        self.samples = []
        self.max_mhz = None
        self.error = None

    def _sample(self):
        self.samples.append((self.nvml.sm_clock(self.h), self.nvml.reasons(self.h)))

    def _run(self):
        while not self.stop.wait(0.005):
            try:
                self._sample()
            except Exception:
                return

    def __enter__(self):
        import threading

        import torch

        try:
            self.nvml = _Nvml()
            pr = torch.cuda.get_device_properties(self.dev)
            try:  # the CUDA device by its PCI address (NVML and CUDA may order devices differently)
                bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            except AttributeError:
                bus = None
            self.h = self.nvml.handle(bus, self.dev)
            self.max_mhz = self.nvml.sm_max(self.h)
            self._sample()
            self.stop = threading.Event()
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        except Exception as e:  # no NVML: the line reports no samples and why
            self.h = None
            self.error = f"{type(e).__name__}: {e}"
        return self

    def __exit__(self, *a):
        if self.h is None:
            return
        self.stop.set()
        self.t.join(timeout=1.0)
        try:
            self._sample()
        except Exception:
            pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "error": self.error}
        reasons = sorted({n for _, r in self.samples for n, bit in self.REASONS if r & bit})
        return {"sm_mhz": statistics.median(sm for sm, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples), "source": "NVML, every 5 ms"}


def _rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


# ---------------------------------------------------------------- workloads on the device
class _Workload:
    """Device state and the step of one configuration."""

    def __init__(self, cfg, dev):
        import torch

        from paper_2505_22313_b300 import _lib, api, inputs
        from paper_2505_22313_b300.api import Geometry

        self.cfg, self.dev = cfg, dev
        N = cfg["N"]
        P = PAD * N
        self.N, self.P = N, P
        f = cfg.get("upsample", 1)
        self.NL = N // f
        self.g = Geometry.make(N, cfg["dx"], cfg["z"], cfg["lambdas"], n_index=N_INDEX, pad=PAD, upsample=f)
        S = self.g.L
        # heights (on the (N / f)^2 layout): the numpy recipe up to 8192^2; the device generator
        # (same recipe, torch's RNG) for the 32768^2 large-area map, which the host would take a
        # minute to smooth
        if self.NL <= 8192:
            self.h_np = inputs.heights(self.NL, cfg["h_seed"])
            self.h = torch.from_numpy(self.h_np).to(dev)
        else:
            self.h = inputs.heights_device(self.NL, cfg["h_seed"], dev)
            self.h_np = None
        grad = "grad" in cfg["step"]
        self.ws = api.workspace(api.workspace_bytes(self.g, _lib.DOE_OP_GRAD if grad else _lib.DOE_OP_PSF), dev)
        self.psf = torch.empty((S, P, P), dtype=torch.float32, device=dev)
        self.kmax = [int(k) for k in api.band_limits(self.g)[0]]
        if "render" in cfg["step"]:
            C, H, W = cfg["C"], cfg["H"], cfg["W"]
            self.img_np = inputs.image(C, H, W, cfg["img_seed"])
            self.img = torch.from_numpy(self.img_np).to(dev)
            self.ws_r = api.workspace(_lib.load().doe_render_workspace_bytes(C, H, W), dev)
            self.out = torch.empty((C, H, W), dtype=torch.float32, device=dev)
        if grad:
            self.T = inputs.spot_target_device(P, N, S, cfg["tgt_seed"], dev)
            self.gr = torch.empty((self.NL, self.NL), dtype=torch.float32, device=dev)
            self.loss = torch.empty((1,), dtype=torch.float64, device=dev)
        self.units = S * P * P

    def step(self, h=None, stream=None):
        from paper_2505_22313_b300 import api

        h = self.h if h is None else h
        api.psf(h, self.g, out=self.psf, ws=self.ws, stream=stream)
        if "render" in self.cfg["step"]:
            api.render(self.psf, self.img, out=self.out, ws=self.ws_r, stream=stream)
        if "grad" in self.cfg["step"]:
            api.grad(h, self.g, self.T, ws=self.ws, out=self.gr, loss=self.loss, recompute=True, stream=stream)

    def alg(self):
        c = self.cfg
        return (_algorithmic_bytes(self.kmax, self.P, self.N, c.get("C", 0), c.get("H", 0), c.get("W", 0), self.NL),
                _algorithmic_flops(self.kmax, self.P, self.N, c.get("C", 0), c.get("H", 0), c.get("W", 0)))


def _time_steps(wl, K, W, dev, ws_n, flush=False):
    """W warm-up steps, then K timed steps between barriers and synchronizes, each bracketed
    by CUDA events on the launching stream, with per-pass events from the library."""
    import torch
    import torch.distributed as dist

    from paper_2505_22313_b300 import api
    from paper_2505_22313_b300.replicas import max_over_ranks

    for _ in range(W):
        wl.step()
    torch.cuda.synchronize()
    scratch = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if flush else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    api.trace_enable(K * 24)
    n0 = api.launch_count()
    if ws_n > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with _Clocks(dev.index if dev.index is not None else 0) as clk:
        t0 = time.perf_counter()
        for k in range(K):
            if scratch is not None:
                scratch.fill_(k & 255)  # evicts the previous step's data from L2 (outside the step's events)
            ev[k][0].record()
            wl.step()
            ev[k][1].record()
        torch.cuda.synchronize()
        if ws_n > 1:
            dist.barrier()
        wall = time.perf_counter() - t0
    launches = api.launch_count() - n0
    recs = api.trace_read(K * 24)
    api.trace_enable(0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(ev[0][0].elapsed_time(ev[-1][1]))
    if flush:  # the region includes the flushes: take the steps' own time
        total_ms = max_over_ranks(sum(step_ms))
    per = {}
    for name, ms in recs:
        per.setdefault(name, []).append(ms)
    return dict(total_ms=total_ms, step_ms=step_ms, per=per, launches=launches, clk=clk.summary(), wall=wall)


def _roofline(wl, t, dev, workload):
    alg, flops = wl.alg()
    per = t["per"]
    # the dominant pass among those with algorithmic bytes (a table set-up pass has none)
    dom = max((k for k in per if alg.get(k)), key=lambda k: sum(per[k]))
    avg_ms = sum(per[dom]) / len(per[dom])
    peak, peak_kind = _peaks()
    achieved = alg[dom] / (avg_ms / 1e3) / 1e9
    alu_peak, alu_src = _fp32_peak_tflops(dev, t["clk"])
    alu = flops[dom] / (avg_ms / 1e3) / 1e12
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
            "traffic": _traffic(workload, dom), "algorithmic_bytes_per_launch": alg[dom],
            "avg_launch_ms": round(avg_ms, 4),
            "passes_ms": {k: round(sum(v) / len(v), 4) for k, v in per.items()},
            "pass_hbm_frac": {k: round(alg[k] / (sum(v) / len(v) / 1e3) / 1e9 / peak, 4) for k, v in per.items()
                              if k in alg and alg[k]},
            "alu": {"achieved": round(alu, 2), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                    "frac": round(alu / alu_peak, 4), "flops_per_launch": flops[dom],
                    "convention": "5 n log2 n per length-n complex transform + pointwise products; peak = " + alu_src}}


def _fp64_rows_check(wl, j, rows):
    """Relative L2 error of wavelength j's PSF on the given rows against the FP64 oracle's
    row-subset mode.  Returns (error, seconds)."""
    import oracle

    import oracle as _o

    h = wl.h_np if wl.h_np is not None else wl.h.cpu().numpy()
    f = wl.cfg.get("upsample", 1)
    if f > 1:
        h = _o.upsample_nearest(h, f)
    t0 = time.perf_counter()
    lam = wl.cfg["lambdas"][j]
    if len(rows) == wl.P:
        ref = oracle.psf(h, wl.cfg["dx"], wl.cfg["z"], [lam], n_index=N_INDEX, pad=PAD)[0]
        got = wl.psf[j].cpu().numpy()
    else:
        ref = oracle.psf_rows(h, wl.cfg["dx"], wl.cfg["z"], lam, np.asarray(rows), n_index=N_INDEX, pad=PAD)
        import torch

        got = wl.psf[j][torch.as_tensor(rows, device=wl.psf.device)].cpu().numpy()
    return _rel_l2(got, ref), time.perf_counter() - t0


def _sub_record(c, dev, K, W, check=True):
    """One configuration measured on its own: step time, per-pass times, dominant pass's
    roofline, clocks, FP64 error on oracle rows."""
    import torch

    cfg = CONFIGS[c]
    wl = _Workload(cfg, dev)
    flush = c == 1
    t = _time_steps(wl, K, W, dev, 1, flush=flush)
    srt = sorted(t["step_ms"])
    ms = statistics.median(t["step_ms"]) if flush else t["total_ms"] / K
    rec = {"workload": cfg["workload"], "config": _config(cfg), "steps": K, "warmup": W,
           "value": wl.units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
           "roofline": _roofline(wl, t, dev, cfg["workload"]), "clocks": t["clk"], "gpu_launches": t["launches"]}
    if "grad" in cfg["step"]:
        rec["loss"] = float(wl.loss.item())
    if check:
        P = wl.P
        j = len(cfg["lambdas"]) // 2
        rows = list(range(P)) if P <= 8192 else sorted({0, P // 8, P // 2 - 1, P // 2, 5 * P // 8, P - 1})
        err, secs = _fp64_rows_check(wl, j, rows)
        rec["fp64_rel_l2_psf"] = {"value": err, "wavelength_nm": round(cfg["lambdas"][j] * 1e9, 1),
                                  "rows": "all" if len(rows) == P else rows, "oracle_s": round(secs, 1)}
    del wl
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def _serving_record(dev, n_requests=None):
    """A seeded Poisson trace through the continuous-batching scheduler and through the
    one-request-at-a-time baseline (the same kernels, one wavelength per launch, synchronous),
    heights uploaded per request from pinned host memory."""
    import torch

    from paper_2505_22313_b300 import inputs
    from paper_2505_22313_b300.serve import (CudaLauncher, HostHeights, Scheduler, serve_one_at_a_time,
                                             trace_from_stream)

    s = SERVING
    n = n_requests or s["requests"]
    trace = trace_from_stream(inputs.request_stream(n, s["rate_hz"], seed=s["seed"], sides=s["sides"],
                                                    max_lambda=s["max_lambda"]))
    hsrc = HostHeights(s["sides"], device=dev)
    base, _ = serve_one_at_a_time(trace, device=dev, heights_source=hsrc)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    budget = 140 << 30
    lau = CudaLauncher(n_streams=3, ws_bytes=20 << 30, device=dev, psf_arena_bytes=budget, heights_source=hsrc)
    with _Clocks(dev.index if dev.index is not None else 0) as clk:
        st = Scheduler(lau, budget).run(trace)
        torch.cuda.synchronize()
    b, o = st.summary(), base.summary()
    del lau
    torch.cuda.empty_cache()
    return {"workload": s["workload"],
            "config": {"requests": n, "rate_hz": s["rate_hz"], "sides": list(s["sides"]), "max_lambda": s["max_lambda"],
                       "z_mm": [10, 100], "pitch_um": 1.0, "budget_gb": 140, "streams": 3,
                       "heights": "one seeded map per side in pinned host memory, uploaded per request"},
            "value": b["samples_per_s"], "unit": UNIT, "batched": b, "one_at_a_time": o,
            "speedup_vs_one_at_a_time": (b["samples_per_s"] / o["samples_per_s"]) if o["samples_per_s"] else None,
            "clocks": clk.summary()}


def _oracle_sample(h, lams, img1, psf_gpu=None, j_cmp=0):
    """FP64 oracle on a bounded sample of the RGB workload: the 8192^2 PSFs of `lams` and one
    render channel.  Returns (seconds, threads, rel L2 error of the GPU PSF of wavelength
    j_cmp if given)."""
    import oracle

    t0 = time.perf_counter()
    ref = oracle.psf(h, WL["dx"], WL["z"], lams, n_index=N_INDEX, pad=PAD)
    oracle.render(ref[:1].astype(np.float32), img1)
    dt = time.perf_counter() - t0
    err = None
    if psf_gpu is not None:
        err = _rel_l2(psf_gpu, ref[j_cmp])
    return dt, oracle.num_threads(), err


def _e2e(wl, K, dev, ws_n):
    """End to end through the public API: pinned host inputs in, the step's result out, every
    step; copy-in, compute and copy-out on three streams with two buffer slots, so one step's
    copies overlap its neighbours' kernels (as a design loop fed from host memory would run).
    Inputs: the heights (and the image of the render step); result: the rendered image or the
    gradient and loss."""
    import torch

    from paper_2505_22313_b300.replicas import max_over_ranks

    render = "render" in wl.cfg["step"]
    h_host = wl.h.cpu().pin_memory()
    ins = [(h_host, [wl.h, torch.empty_like(wl.h)])]
    if render:
        ins.append((torch.from_numpy(wl.img_np).pin_memory(), [wl.img, torch.empty_like(wl.img)]))
    res = wl.out if render else wl.gr
    out_host = [torch.empty(res.shape, dtype=res.dtype).pin_memory() for _ in range(2)]
    out_dev = [res, torch.empty_like(res)]
    loss_host = [torch.empty((1,), dtype=torch.float64).pin_memory() for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    cmp_done = [torch.cuda.Event() for _ in range(2)]
    in_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    for b in range(2):  # slots start free
        cmp_done[b].record(s_cmp)
        out_done[b].record(s_out)
    img_keep = wl.img if render else None
    gr_keep = wl.gr if not render else None

    def step_e2e(k):
        b = k % 2
        s_in.wait_event(cmp_done[b])  # the step that last read this input slot has finished
        with torch.cuda.stream(s_in):
            for host, slots in ins:
                slots[b].copy_(host, non_blocking=True)
            in_done[b].record(s_in)
        s_cmp.wait_event(in_done[b])
        s_cmp.wait_event(out_done[b])  # this output slot has been copied out
        if render:
            wl.img = ins[1][1][b]
            wl.out = out_dev[b]
        else:
            wl.gr = out_dev[b]
        wl.step(h=ins[0][1][b], stream=s_cmp)
        cmp_done[b].record(s_cmp)
        s_out.wait_event(cmp_done[b])
        with torch.cuda.stream(s_out):
            out_host[b].copy_(out_dev[b], non_blocking=True)
            if not render:
                loss_host[b].copy_(wl.loss, non_blocking=True)
            out_done[b].record(s_out)

    for k in range(4):
        step_e2e(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(K):
        step_e2e(k)
    e1.record(s_out)  # after the last copy-out, which follows every earlier step's work
    torch.cuda.synchronize()
    if render:
        wl.img, wl.out = img_keep, out_dev[0]
    else:
        wl.gr = gr_keep
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / K)
    h2d = sum(host.numel() * host.element_size() for host, _ in ins)
    d2h = res.numel() * res.element_size() + (0 if render else 8)
    return {"value": ws_n * wl.units / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4), "steps": K,
            "overlap": "copy-in / compute / copy-out streams, 2 slots"}


def _cufft_comparison(wl, dev):
    """The unfused cuFFT chain on the same GPU (comparison only; libdoe does not use cuFFT)."""
    import ctypes

    import torch

    from paper_2505_22313_b300 import api
    from paper_2505_22313_b300 import build as _b

    try:
        clib = ctypes.CDLL(str(_b.COMPARE_LIB))
        clib.doe_cufft_psf.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_size_t, ctypes.c_void_p]
        clib.doe_cufft_psf.restype = ctypes.c_int
        P = wl.P
        cws = api.workspace(P * P * 8, dev)
        cpsf = torch.empty_like(wl.psf)
        gc = wl.g.c()
        s_ = torch.cuda.current_stream()

        def cstep():
            rc = clib.doe_cufft_psf(ctypes.byref(gc), ctypes.c_void_p(wl.h.data_ptr()), ctypes.c_void_p(cpsf.data_ptr()),
                                    ctypes.c_void_p(cws.data_ptr()), cws.numel(), ctypes.c_void_p(s_.cuda_stream))
            assert rc == 0, rc

        for _ in range(3):
            cstep()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(10):
            cstep()
        a1.record()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        for _ in range(10):
            api.psf(wl.h, wl.g, out=wl.psf, ws=wl.ws)
        b1.record()
        torch.cuda.synchronize()
        diff = (torch.linalg.vector_norm((cpsf - wl.psf).double()) / torch.linalg.vector_norm(wl.psf.double())).item()
        out = {"psf_ms": round(a0.elapsed_time(a1) / 10, 4), "ours_psf_ms": round(b0.elapsed_time(b1) / 10, 4),
               "rel_l2_vs_ours": diff}
        del cws, cpsf
        return out
    except (OSError, AttributeError, AssertionError) as exc:
        return {"unavailable": str(exc)[:200]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2505_22313_b300 import api, build

    ws_n, rank, local = _dist()
    if ws_n > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    api.init()

    main_c = args.config or 2
    if main_c == 5:
        if rank == 0:
            rec = _serving_record(dev, args.requests)
            line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
                    "ms_per_step": rec["batched"]["makespan_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": rec["config"] | {"workload": rec["workload"]},
                    "serving": rec, "clocks": rec["clocks"]}
            print(json.dumps(line), flush=True)
        return
    cfg = CONFIGS[main_c]
    K = args.steps
    wl = _Workload(cfg, dev)
    t = _time_steps(wl, K, args.warmup, dev, ws_n, flush=main_c == 1)
    ms = statistics.median(t["step_ms"]) if main_c == 1 else t["total_ms"] / K
    value = ws_n * wl.units / (ms / 1e3)
    roof = _roofline(wl, t, dev, cfg["workload"])
    e2e = _e2e(wl, max(3, min(K, 50 if wl.P <= 16384 else 5)), dev, ws_n)
    cufft = _cufft_comparison(wl, dev) if main_c == 2 else None

    cpu = None
    fp64_err = None
    if rank == 0 and ws_n == 1 and not args.no_cpu_baseline:
        if main_c == 2:
            psf1 = wl.psf[1].cpu().numpy()
            dt, cores, fp64_err = _oracle_sample(wl.h_np, list(cfg["lambdas"]), wl.img_np[1:2], psf1, j_cmp=1)
            cpu = {"value": len(cfg["lambdas"]) * wl.P * wl.P / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "FP64 oracle: the three 8192^2 PSFs of one step (450/550/650 nm) and one 2048^2 render "
                             f"channel ({dt:.1f} s)"}
        else:
            import oracle

            j = len(cfg["lambdas"]) // 2
            rows = list(range(wl.P)) if wl.P <= 8192 else sorted({0, wl.P // 8, wl.P // 2 - 1, wl.P // 2, 5 * wl.P // 8, wl.P - 1})
            fp64_err, dt = _fp64_rows_check(wl, j, rows)
            cpu = {"value": wl.P * wl.P / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"FP64 oracle: the {wl.P}^2 PSF of one wavelength "
                             f"({'full' if wl.P <= 8192 else 'row-subset mode, every sample transformed'}, {dt:.1f} s)"}
    subs = None
    if rank == 0 and ws_n == 1 and args.config is None and not args.no_sub:
        del wl
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        subs = {}
        for c, k in SUBS:
            subs[f"c{c}" if isinstance(c, int) else c] = _sub_record(c, dev, min(K, k), 3, check=not args.no_cpu_baseline)
        subs["c5"] = _serving_record(dev)
    if ws_n > 1:
        dist.barrier()
    if rank != 0:
        if ws_n > 1:
            dist.destroy_process_group()
        return
    srt = sorted(t["step_ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": _config(cfg, {"parallelism": f"replicas x{ws_n}" if ws_n > 1 else "single GPU"}),
        "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
        f"fp64_rel_l2_psf_{round(cfg['lambdas'][len(cfg['lambdas']) // 2] * 1e9)}nm": fp64_err,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": t["clk"], "gpu_launches": t["launches"],
        "cufft_chain_comparison": cufft, "configs": subs, "wall_s": round(t["wall"], 3),
    }
    print(json.dumps(line), flush=True)
    if ws_n > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step a bounded sample of the workload
    (the PSF of one wavelength, plus one render channel for the RGB workload) on the host
    cores.  A sample takes ~10 s on 16 cores at the RGB workload, so the arm runs at most as
    many steps as fit in ~200 s and reports both the requested and the executed step counts;
    warm-up is skipped (the oracle has nothing to warm)."""
    ws_n, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2505_22313_b300 import inputs

    c = args.config or 2
    if c == 5:
        c = 2  # the serving trace has no oracle arm of its own: its unit of work is the RGB workload's
    cfg = CONFIGS[c]
    N, P = cfg["N"], PAD * cfg["N"]
    j = len(cfg["lambdas"]) // 2
    lam = cfg["lambdas"][j]
    f = cfg.get("upsample", 1)
    if N // f > 8192:
        h_np = inputs.heights_device(N // f, cfg["h_seed"], "cpu").numpy()
    else:
        h_np = inputs.heights(N // f, cfg["h_seed"])
    if f > 1:
        h_np = oracle.upsample_nearest(h_np, f)
    img1 = inputs.image(cfg["C"], cfg["H"], cfg["W"], cfg["img_seed"])[1:2] if "render" in cfg["step"] else None
    rows = np.array(sorted({0, P // 8, P // 2 - 1, P // 2, 5 * P // 8, P - 1}))
    times = []
    budget_s = 200.0
    while len(times) < args.steps:
        t0 = time.perf_counter()
        if P <= 8192:
            ref = oracle.psf(h_np, cfg["dx"], cfg["z"], [lam], n_index=N_INDEX, pad=PAD)
            if img1 is not None:
                oracle.render(ref[:1].astype(np.float32), img1)
        else:
            oracle.psf_rows(h_np, cfg["dx"], cfg["z"], lam, rows, n_index=N_INDEX, pad=PAD)
        dt = time.perf_counter() - t0
        times.append(dt)
        if sum(times) + dt > budget_s:
            break
    tot = sum(times)
    value = P * P * len(times) / tot
    srt = sorted(times)
    sample = (f"FP64 oracle, per step: the {P}^2 PSF of one wavelength ({lam * 1e9:.0f} nm)"
              + (" and one 2048^2 render channel" if img1 is not None else "")
              + ("" if P <= 8192 else " in row-subset mode (every sample transformed, 6 output rows kept)"))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": len(times),
        "steps_requested": args.steps, "warmup": 0, "warmup_requested": args.warmup,
        "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(cfg, {"parallelism": "host cores"}),
        "latency_ms": {"p50": 1e3 * srt[len(srt) // 2], "p99": 1e3 * srt[-1]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default=None, choices=["1", "2", "3", "4", "5", *[k for k in CONFIGS if isinstance(k, str)]],
                    help="run this workload as the main line (default: the RGB design evaluation with sub-records)")
    ap.add_argument("--requests", type=int, default=None, help="serving trace length (--config 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing and error checks")
    ap.add_argument("--no-sub", action="store_true", help="skip the per-configuration sub-records")
    ap.add_argument("--ingest-traffic", metavar="CSV", default=None,
                    help="write profiles/traffic.json from an ncu CSV of the PSF + render step and exit")
    ap.add_argument("--ncu-command", default="", help="the ncu command that wrote the CSV (recorded with it)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    if args.config is not None and args.config.isdigit():
        args.config = int(args.config)
    if args.ingest_traffic:
        wl = CONFIGS[args.config if args.config is not None else 2]["workload"]
        print(json.dumps(ingest_traffic(args.ingest_traffic, wl, args.ncu_command)["workloads"][wl], indent=1))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
