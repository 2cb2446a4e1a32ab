"""Continuous-batching server for DOE evaluations (PSFs of many independent requests).

A request is one DOE (side N, padded P = 2N) with its own wavelengths and distance.  Its work
is split into units of a few wavelengths each.  The scheduler:
  * admits arrived requests in FIFO order while their device footprint (heights + PSFs)
    fits the HBM budget; admitted requests keep all their state on the device;
  * forms launches from pending units of one grid size P (oldest pending unit first), up to
    64 wavelengths or the per-stream workspace, so one set of kernels serves several
    requests (doe_psf_many); requests that arrive while others run are admitted as memory
    frees up;
  * routes launches by grid size: one launch of a large grid (P >= 16384) fills the GPU, so
    large-grid launches queue back to back on one stream in arrival order (served at full
    speed, none time-shared with another large one), while smaller grids run on the other
    streams beside them; small work also takes the large lane when no large work waits;
  * polls completion events without blocking and with a host deadline per request
    (a request past its deadline is reported as timed out, DOE_ETIMEDOUT);
  * hands each finished request to a consumer callback, which frees its PSFs.
The scheduler is plain host logic; the device side lives in CudaLauncher, so the logic can be
tested with a fake launcher and a fake clock.  The baseline serve_one_at_a_time() runs the
same kernels with one wavelength per launch, synchronously, in arrival order.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

DOE_ETIMEDOUT = -5
DOE_ENOMEM = -7  # serving: request larger than the admission budget


@dataclass
class Req:
    rid: int
    arrival_s: float
    N: int
    lambdas: np.ndarray
    z: float
    dx: float = 1e-6
    seed: int = 0
    n_index: float = 1.46
    deadline_s: float = float("inf")  # relative to arrival

    @property
    def P(self) -> int:
        return 2 * self.N

    @property
    def L(self) -> int:
        return int(len(self.lambdas))

    def footprint(self) -> int:
        """Device bytes held while admitted: heights + PSFs."""
        return 4 * self.N * self.N + 4 * self.L * self.P * self.P

    def samples(self) -> int:
        return self.L * self.P * self.P


@dataclass
class Unit:
    req: Req
    j0: int  # first wavelength index
    j1: int  # one past the last


@dataclass
class Stats:
    latency_s: dict = field(default_factory=dict)
    status: dict = field(default_factory=dict)
    launches: int = 0
    peak_bytes: int = 0
    makespan_s: float = 0.0
    samples: int = 0

    def summary(self) -> dict:
        lat = sorted(v for k, v in self.latency_s.items() if self.status.get(k, 0) == 0)
        pct = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
        return {"requests": len(self.status), "completed": len(lat),
                "timed_out": sum(1 for s in self.status.values() if s == DOE_ETIMEDOUT),
                "p50_s": pct(0.50), "p99_s": pct(0.99), "makespan_s": self.makespan_s,
                "samples_per_s": self.samples / self.makespan_s if self.makespan_s > 0 else None,
                "launches": self.launches, "peak_admitted_bytes": self.peak_bytes}


class Arena:
    """First-fit sub-allocator of byte ranges in one pre-allocated device buffer, so admitting
    a request never calls the device allocator.  Ranges are 256-byte aligned; freed ranges
    coalesce with their neighbours."""

    ALIGN = 256

    def __init__(self, nbytes: int):
        self.size = int(nbytes)
        self.free = [(0, self.size)]  # sorted, disjoint (offset, length)
        self.used = 0

    def _round(self, n: int) -> int:
        return (int(n) + self.ALIGN - 1) // self.ALIGN * self.ALIGN

    def fits(self, n: int) -> bool:
        n = self._round(n)
        return any(length >= n for _, length in self.free)

    def alloc(self, n: int) -> int | None:
        n = self._round(n)
        for i, (off, length) in enumerate(self.free):
            if length >= n:
                if length == n:
                    del self.free[i]
                else:
                    self.free[i] = (off + n, length - n)
                self.used += n
                return off
        return None

    def release(self, off: int, n: int) -> None:
        n = self._round(n)
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, n))
        self.used -= n
        # coalesce with the following and the preceding range
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]


class Scheduler:
    """Continuous batching with admission by device-memory footprint.

    launcher: object with
        n_slots                      -- launch slots (a slot holds one launch in flight)
        lanes (optional)             -- per slot "large", "small" or "any" (default: all "any")
        ws_bytes(units) -> int       -- workspace one launch of these units needs
        ws_limit                     -- workspace available per slot
        admit(req), release(req)     -- allocate / free a request's device state
        fits(req) (optional)         -- whether admit(req) can place the request now
        launch(slot, units)          -- enqueue the units' PSFs on the slot's stream
        done(slot) -> bool           -- non-blocking completion test of the slot's last launch
    clock: callable returning seconds."""

    MAX_SLICES = 64

    def __init__(self, launcher, budget_bytes: int, clock=time.perf_counter, unit_lambdas: int = 8,
                 consumer=None, large_P: int = 16384):
        self.L = launcher
        self.large_P = int(large_P)
        self.budget = int(budget_bytes)
        self.clock = clock
        self.unit_lambdas = unit_lambdas
        self.consumer = consumer

    def _split(self, r: Req) -> list[Unit]:
        out = []
        j = 0
        while j < r.L:
            j1 = min(r.L, j + self.unit_lambdas)
            while j1 > j + 1 and self.L.ws_bytes([Unit(r, j, j1)]) > self.L.ws_limit:
                j1 -= 1
            out.append(Unit(r, j, j1))
            j = j1
        return out

    def run(self, trace: list[Req], poll_sleep_s: float = 0.0) -> Stats:
        st = Stats()
        arrivals = collections.deque(sorted(trace, key=lambda r: (r.arrival_s, r.rid)))
        waiting: collections.deque[Req] = collections.deque()
        pending: dict[int, collections.deque[Unit]] = collections.defaultdict(collections.deque)
        remaining: dict[int, int] = {}
        admitted: dict[int, Req] = {}
        used = [0]
        slots: list[list[Unit] | None] = [None] * self.L.n_slots
        n_total = len(arrivals)
        t0 = self.clock()

        def finish(r: Req):
            if r.rid not in st.status:  # completed normally (not timed out)
                st.latency_s[r.rid] = self.clock() - t0 - r.arrival_s
                st.status[r.rid] = 0
                st.samples += r.samples()
                if self.consumer:
                    self.consumer(r)
            self.L.release(r)
            used[0] -= r.footprint()
            del admitted[r.rid]

        while True:
            now = self.clock() - t0
            while arrivals and arrivals[0].arrival_s <= now:
                waiting.append(arrivals.popleft())
            # completions (non-blocking event queries)
            for s, units in enumerate(slots):
                if units is not None and self.L.done(s):
                    slots[s] = None
                    for u in units:
                        remaining[u.req.rid] -= 1
                        if remaining[u.req.rid] == 0:
                            finish(u.req)
            # host deadlines: a request past its deadline is reported as timed out; its unlaunched
            # work is dropped, work already on the device is left to finish, then it is freed
            now = self.clock() - t0
            for r in [r for r in waiting if now - r.arrival_s > r.deadline_s]:
                waiting.remove(r)
                st.status[r.rid] = DOE_ETIMEDOUT
            for rid, r in list(admitted.items()):
                if rid not in st.status and now - r.arrival_s > r.deadline_s:
                    st.status[rid] = DOE_ETIMEDOUT
                    keep = collections.deque(u for u in pending[r.P] if u.req.rid != rid)
                    remaining[rid] -= len(pending[r.P]) - len(keep)
                    pending[r.P] = keep
                    if remaining[rid] == 0:
                        finish(r)
            # admission: FIFO, so a large request at the head is not starved by later small ones;
            # a request larger than the whole budget can never run and is refused
            while waiting:
                r = waiting[0]
                if r.footprint() > self.budget:
                    waiting.popleft()
                    st.status[r.rid] = DOE_ENOMEM
                    continue
                if used[0] + r.footprint() > self.budget:
                    break
                if hasattr(self.L, "fits") and not self.L.fits(r):
                    break  # no contiguous range yet: wait for releases (keeps FIFO order)
                waiting.popleft()
                self.L.admit(r)
                used[0] += r.footprint()
                st.peak_bytes = max(st.peak_bytes, used[0])
                admitted[r.rid] = r
                units = self._split(r)
                remaining[r.rid] = len(units)
                pending[r.P].extend(units)
            # launches into free slots: of the grid-size classes this slot's lane serves, the
            # one holding the oldest pending unit
            lanes = getattr(self.L, "lanes", None) or ["any"] * len(slots)
            for s in range(len(slots)):
                if slots[s] is not None:
                    continue
                live = [(q[0].req.arrival_s, q[0].req.rid, P) for P, q in pending.items() if q]
                if not live:
                    break
                if lanes[s] == "large":
                    cand = [x for x in live if x[2] >= self.large_P]
                    if not cand and not any(slots[k] is not None and lanes[k] == "large" and
                                            slots[k][0].req.P >= self.large_P for k in range(len(slots))):
                        cand = live  # no large work waiting or running: small work may use the lane
                elif lanes[s] == "small":
                    cand = [x for x in live if x[2] < self.large_P]
                else:
                    cand = live
                if not cand:
                    continue
                P = min(cand)[2]
                q = pending[P]
                batch = [q.popleft()]
                while q:
                    nxt = batch + [q[0]]
                    if sum(u.j1 - u.j0 for u in nxt) > self.MAX_SLICES or self.L.ws_bytes(nxt) > self.L.ws_limit:
                        break
                    batch.append(q.popleft())
                self.L.launch(s, batch)
                slots[s] = batch
                st.launches += 1
            if not arrivals and not waiting and not admitted and all(x is None for x in slots):
                break
            if len(st.status) == n_total:  # every request completed, timed out or refused; work
                break                      # of timed-out requests still on the device stays in flight
            if poll_sleep_s:
                time.sleep(poll_sleep_s)
        self.inflight = [u for us in slots if us for u in us]
        st.makespan_s = self.clock() - t0
        return st


class CudaLauncher:
    """Device side of the scheduler: per-stream workspaces, seeded heights generated on the
    device at admission, doe_psf_many launches, completion events.  Stream 0 is the large
    lane: `large_depth` slots queue on it, so its launches run back to back; every other
    stream has one small-lane slot.  Launches on one stream share its workspace (stream order
    keeps them apart)."""

    def __init__(self, n_streams: int = 3, ws_bytes: int = 24 << 30, device=None, keep_results: bool = False,
                 large_depth: int = 2, psf_arena_bytes: int | None = None, heights_source=None):
        import torch

        from . import api
        from .api import Geometry

        self.torch, self.api, self.Geometry = torch, api, Geometry
        self.dev = torch.device(device or "cuda")
        self.ws_limit = int(ws_bytes)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        self.ws = [api.workspace(self.ws_limit, self.dev) for _ in range(n_streams)]
        self.slot_stream = [0] * large_depth + list(range(1, n_streams))
        self.lanes = ["large"] * large_depth + ["small"] * (n_streams - 1)
        self.n_slots = len(self.slot_stream)
        self.events = [None] * self.n_slots
        # heights_source(req) -> the request's heights: a device tensor, or a pinned host tensor
        # copied in on the upload stream (default: seeded heights generated on the device)
        self.heights_source = heights_source
        # heights and PSFs live in one buffer allocated here (None: tensors per request)
        self.arena = Arena(psf_arena_bytes) if psf_arena_bytes else None
        self.arena_buf = torch.empty(psf_arena_bytes, dtype=torch.uint8, device=self.dev) if psf_arena_bytes else None
        self.state: dict[int, tuple] = {}
        self.keep = keep_results
        self.results: dict[int, "torch.Tensor"] = {}
        self.upload = torch.cuda.Stream(self.dev)

    def _geom(self, u: Unit):
        r = u.req
        return self.Geometry.make(r.N, r.dx, r.z, r.lambdas[u.j0:u.j1], n_index=r.n_index)

    def ws_bytes(self, units) -> int:
        import ctypes

        from . import _lib

        gs = [self._geom(u) for u in units]
        arr = (_lib.Geom * len(gs))(*[g.c() for g in gs])
        return int(_lib.load().doe_workspace_bytes_many(len(gs), arr, _lib.DOE_OP_PSF))

    def fits(self, r: Req) -> bool:
        return self.arena is None or self.arena.fits(r.footprint())

    def _heights(self, r: Req):
        if self.heights_source is not None:
            return self.heights_source(r)
        from .inputs import heights_device

        return heights_device(r.N, r.seed, self.dev)

    def admit(self, r: Req):
        torch = self.torch
        off = None
        with torch.cuda.stream(self.upload):
            src = self._heights(r)
            if self.arena is not None:
                # one range: heights [N][N] then PSFs [L][P][P], both float32
                off = self.arena.alloc(r.footprint())
                if off is None:
                    raise MemoryError("serving arena: no contiguous range (admit without fits)")
                hb = 4 * r.N * r.N
                h = self.arena_buf[off:off + hb].view(torch.float32).view(r.N, r.N)
                h.copy_(src, non_blocking=True)
                out = self.arena_buf[off + hb:off + r.footprint()].view(torch.float32).view(r.L, r.P, r.P)
            else:
                h = src if src.device.type == "cuda" else src.to(self.dev, non_blocking=True)
                out = torch.empty((r.L, r.P, r.P), dtype=torch.float32, device=self.dev)
            ev = torch.cuda.Event()
            ev.record(self.upload)
        self.state[r.rid] = (h, out, ev, off, src)

    def release(self, r: Req):
        h, out, _, off, _ = self.state.pop(r.rid)
        if self.keep:
            # the range is reused by later requests: keep a copy, made before it can be
            self.results[r.rid] = out.clone() if off is not None else out
            if off is not None:
                self.torch.cuda.synchronize(self.dev)
        if off is not None:
            self.arena.release(off, r.footprint())

    def launch(self, slot: int, units):
        torch = self.torch
        si = self.slot_stream[slot]
        st = self.streams[si]
        hs, outs, gs = [], [], []
        for u in units:
            h, out, ev, _, _ = self.state[u.req.rid]
            st.wait_event(ev)
            hs.append(h)
            outs.append(out[u.j0:u.j1])
            gs.append(self._geom(u))
        with torch.cuda.stream(st):
            self.api.psf_many(hs, gs, outs=outs, ws=self.ws[si], stream=st)
            for h, o in zip(hs, outs):
                h.record_stream(st)
                o.record_stream(st)
            e = torch.cuda.Event()
            e.record(st)
        self.events[slot] = e

    def done(self, slot: int) -> bool:
        e = self.events[slot]
        return e is None or e.query()


def serve_one_at_a_time(trace: list[Req], device=None, clock=time.perf_counter, keep_results=False,
                        heights_source=None):
    """Baseline: arrival order, one wavelength per doe_psf launch, synchronous (heights from
    heights_source(req) as in CudaLauncher, default seeded on the device)."""
    import torch

    from . import api
    from .api import Geometry
    from .inputs import heights_device

    dev = torch.device(device or "cuda")
    st = Stats()
    results = {}
    ws = None
    t0 = clock()
    for r in sorted(trace, key=lambda r: (r.arrival_s, r.rid)):
        while clock() - t0 < r.arrival_s:
            time.sleep(min(1e-3, max(0.0, r.arrival_s - (clock() - t0))))
        if heights_source is not None:
            h = heights_source(r).to(dev, non_blocking=True)
        else:
            h = heights_device(r.N, r.seed, dev)
        out = torch.empty((r.L, r.P, r.P), dtype=torch.float32, device=dev)
        for j in range(r.L):
            g = Geometry.make(r.N, r.dx, r.z, r.lambdas[j:j + 1], n_index=r.n_index)
            need = api.workspace_bytes(g)
            if ws is None or ws.numel() < need:
                ws = api.workspace(need, dev)
            api.psf(h, g, out=out[j:j + 1], ws=ws)
            torch.cuda.synchronize(dev)
            st.launches += 1
        st.latency_s[r.rid] = clock() - t0 - r.arrival_s
        st.status[r.rid] = 0
        st.samples += r.samples()
        if keep_results:
            results[r.rid] = out
        del out, h
    st.makespan_s = clock() - t0
    return st, results


class HostHeights:
    """Heights as a client would send them: one seeded map per side N (generated once, kept in
    pinned host memory) that every request of that side uploads."""

    def __init__(self, sides, device=None):
        import torch

        from .inputs import heights_device

        dev = torch.device(device or "cuda")
        self.maps = {int(N): heights_device(int(N), 1000 + int(N), dev).cpu().pin_memory() for N in sides}

    def __call__(self, r: Req):
        return self.maps[r.N]


def trace_from_stream(reqs) -> list[Req]:
    """Converts inputs.request_stream() records."""
    return [Req(rid=q.rid, arrival_s=q.arrival_s, N=q.N, lambdas=np.asarray(q.lambdas), z=q.z, dx=q.dx,
                seed=q.seed) for q in reqs]


def main():
    import argparse
    import json
    import os

    # the PSFs of the largest requests are >100 GB tensors: let the caching allocator grow and
    # return segments instead of fragmenting the budget (must be set before CUDA starts)
    os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    import torch

    from . import api, inputs

    ap = argparse.ArgumentParser(description="serving benchmark: continuous batching vs one request at a time")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sides", default="1024,2048,4096,8192,16384")
    ap.add_argument("--max-lambda", type=int, default=31)
    ap.add_argument("--budget-gb", type=float, default=140.0)
    ap.add_argument("--ws-gb", type=float, default=20.0)
    ap.add_argument("--streams", type=int, default=3)
    ap.add_argument("--large-p", type=int, default=16384, help="grids of at least this side use the large lane")
    ap.add_argument("--no-baseline", action="store_true", help="skip the one-request-at-a-time run")
    args = ap.parse_args()
    api.init()
    sides = tuple(int(s) for s in args.sides.split(","))
    trace = trace_from_stream(inputs.request_stream(args.requests, args.rate, sides=sides, max_lambda=args.max_lambda))
    hsrc = HostHeights(sides)
    base = None
    if not args.no_baseline:
        base, _ = serve_one_at_a_time(trace, heights_source=hsrc)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    lau = CudaLauncher(n_streams=args.streams, ws_bytes=int(args.ws_gb * (1 << 30)),
                       psf_arena_bytes=int(args.budget_gb * (1 << 30)), heights_source=hsrc)
    sched = Scheduler(lau, int(args.budget_gb * (1 << 30)), large_P=args.large_p)
    st = sched.run(trace)
    torch.cuda.synchronize()
    print(json.dumps({"trace": {"requests": args.requests, "rate_hz": args.rate, "sides": sides,
                                "max_lambda": args.max_lambda},
                      "scheduler": {"streams": args.streams, "large_p": args.large_p, "budget_gb": args.budget_gb,
                                    "ws_gb": args.ws_gb},
                      "batched": st.summary(), "one_at_a_time": base.summary() if base else None}))


if __name__ == "__main__":
    main()
