"""Host-side tests of the serving scheduler with a fake launcher and a fake clock (no GPU):
admission never exceeds the memory budget, FIFO admission, launch sharing across requests
of equal grid size, latency accounting, bounded waits (timeouts) and refusal of requests
larger than the budget."""
import numpy as np

from paper_2505_22313_b300.serve import DOE_ENOMEM, DOE_ETIMEDOUT, Req, Scheduler


class FakeClock:
    def __init__(self, dt=1e-4):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeLauncher:
    def __init__(self, clock, n_slots=2, ws_limit=1 << 40, sec_per_sample=1e-9, never_done=False):
        self.clock, self.n_slots, self.ws_limit = clock, n_slots, ws_limit
        self.spp, self.never = sec_per_sample, never_done
        self.fin = [None] * n_slots
        self.admitted, self.order, self.batches = set(), [], []

    def ws_bytes(self, units):
        return sum(u.req.P * u.req.P * 8 * (u.j1 - u.j0) for u in units)

    def admit(self, r):
        self.admitted.add(r.rid)
        self.order.append(r.rid)

    def release(self, r):
        self.admitted.remove(r.rid)

    def launch(self, slot, units):
        self.batches.append([(u.req.rid, u.j0, u.j1) for u in units])
        n = sum((u.j1 - u.j0) * u.req.P ** 2 for u in units)
        self.fin[slot] = self.clock() + n * self.spp

    def done(self, slot):
        return (not self.never) and self.fin[slot] is not None and self.clock() >= self.fin[slot]


def _trace(n=40, seed=0, sides=(64, 128, 256), rate=500.0, deadline=float("inf")):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1 / rate)
        out.append(Req(rid=i, arrival_s=t, N=int(rng.choice(sides)),
                       lambdas=rng.uniform(4e-7, 7e-7, int(rng.integers(1, 9))), z=0.05, deadline_s=deadline))
    return out


def test_all_complete_budget_respected_fifo():
    clk = FakeClock()
    trace = _trace()
    budget = 6 * max(r.footprint() for r in trace)
    lau = FakeLauncher(clk)
    st = Scheduler(lau, budget, clock=clk).run(trace)
    s = st.summary()
    assert s["completed"] == len(trace) and s["timed_out"] == 0
    assert st.peak_bytes <= budget
    assert lau.order == sorted(lau.order)  # admitted in arrival order
    assert all(v >= 0 for v in st.latency_s.values())
    assert not lau.admitted  # everything released


def test_launches_are_shared_across_requests():
    clk = FakeClock()
    trace = _trace(n=30, sides=(128,), rate=1e6)  # all arrive at once, same grid size
    lau = FakeLauncher(clk, n_slots=1)
    st = Scheduler(lau, 1 << 40, clock=clk, unit_lambdas=8).run(trace)
    assert st.launches < len(trace)
    assert any(len({rid for rid, _, _ in b}) > 1 for b in lau.batches)
    assert all(sum(j1 - j0 for _, j0, j1 in b) <= Scheduler.MAX_SLICES for b in lau.batches)


def test_timeouts_do_not_hang():
    clk = FakeClock(dt=1e-3)
    trace = _trace(n=6, deadline=0.05)
    lau = FakeLauncher(clk, never_done=True)
    st = Scheduler(lau, 1 << 40, clock=clk).run(trace)
    # the device work never completes: every request is reported as timed out and run() returns
    assert len(st.status) == len(trace)
    assert all(v == DOE_ETIMEDOUT for v in st.status.values())
    assert clk.t < 10.0


def test_oversize_request_refused():
    clk = FakeClock()
    trace = _trace(n=5)
    big = Req(rid=99, arrival_s=0.0, N=4096, lambdas=np.full(3, 5e-7), z=0.05)
    lau = FakeLauncher(clk)
    st = Scheduler(lau, 10 * max(r.footprint() for r in trace), clock=clk).run(trace + [big])
    assert st.status[99] == DOE_ENOMEM
    assert sum(1 for v in st.status.values() if v == 0) == len(trace)


class LaneLauncher(FakeLauncher):
    """Two large-lane slots and one small-lane slot; records the slot of every launch."""

    lanes = ["large", "large", "small"]

    def __init__(self, clock):
        super().__init__(clock, n_slots=3)
        self.slot_of = []

    def launch(self, slot, units):
        super().launch(slot, units)
        self.slot_of.append((slot, units[0].req.P))


def test_large_grids_use_the_large_lane_only():
    clk = FakeClock()
    trace = _trace(n=40, sides=(64, 128, 256), rate=2000.0)
    lau = LaneLauncher(clk)
    st = Scheduler(lau, 1 << 40, clock=clk, large_P=256).run(trace)  # P = 512 is "large"
    assert st.summary()["completed"] == len(trace)
    assert any(P >= 256 for _, P in lau.slot_of) and any(P < 256 for _, P in lau.slot_of)
    for slot, P in lau.slot_of:
        if P >= 256:
            assert LaneLauncher.lanes[slot] == "large"
    # small work reaches the large lane only when no large work waits: with the large requests
    # removed, every slot serves small grids
    lau2 = LaneLauncher(clk)
    Scheduler(lau2, 1 << 40, clock=clk, large_P=1 << 20).run(_trace(n=40, sides=(64, 128), rate=2000.0))
    assert {s for s, _ in lau2.slot_of} >= {0, 2}


def test_arena_first_fit_and_coalescing():
    from paper_2505_22313_b300.serve import Arena

    a = Arena(10 * 256)
    x = a.alloc(256)
    y = a.alloc(300)        # rounds up to 512
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768) and a.used == 1024
    assert a.alloc(2000) is None and not a.fits(2000) and a.fits(1536)
    a.release(y, 300)
    assert a.alloc(512) == 256  # first fit reuses the hole
    a.release(256, 512)
    a.release(x, 256)
    a.release(z, 256)
    assert a.free == [(0, 10 * 256)] and a.used == 0  # everything coalesced


class ArenaLauncher(FakeLauncher):
    """Places each request's PSFs in an Arena; admission asks fits()."""

    def __init__(self, clock, nbytes):
        from paper_2505_22313_b300.serve import Arena

        super().__init__(clock, n_slots=2)
        self.arena = Arena(nbytes)
        self.off = {}

    def fits(self, r):
        return self.arena.fits(r.footprint())

    def admit(self, r):
        super().admit(r)
        self.off[r.rid] = self.arena.alloc(r.footprint())
        assert self.off[r.rid] is not None

    def release(self, r):
        super().release(r)
        self.arena.release(self.off.pop(r.rid), r.footprint())


def test_admission_waits_for_a_contiguous_range():
    clk = FakeClock()
    trace = _trace(n=60, sides=(64, 128, 256), rate=5000.0)
    biggest = max(r.footprint() for r in trace)
    lau = ArenaLauncher(clk, 3 * biggest)
    st = Scheduler(lau, 3 * biggest, clock=clk).run(trace)
    assert st.summary()["completed"] == len(trace)
    assert lau.order == sorted(lau.order)
    assert lau.arena.used == 0 and lau.arena.free == [(0, lau.arena.size)]
