"""Serving on the GPU: each request's PSFs computed in the continuous-batching mix (shared
launches, several streams, admission under a memory budget) equal the same request computed
alone, bit for bit (the kernels are batch-invariant), with PSFs in per-request tensors or in
the launcher's pre-allocated arena, and the one-request-at-a-time baseline gives the same
results."""
import numpy as np
import pytest
import torch

from paper_2505_22313_b300 import api, build
from paper_2505_22313_b300.api import Geometry
from paper_2505_22313_b300.inputs import heights_device
from paper_2505_22313_b300.serve import CudaLauncher, Req, Scheduler, serve_one_at_a_time

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    build.build()
    api.init()


def _trace(n=24, seed=5):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n):
        t += rng.exponential(1e-3)
        out.append(Req(rid=i, arrival_s=t, N=int(rng.choice([64, 128, 256])),
                       lambdas=rng.uniform(4e-7, 7e-7, int(rng.integers(1, 7))), z=float(rng.uniform(1e-3, 2e-2)),
                       seed=7000 + i))
    return out


def _alone(r):
    g = Geometry.make(r.N, r.dx, r.z, r.lambdas, n_index=r.n_index)
    return api.psf(heights_device(r.N, r.seed, "cuda"), g)


@pytest.mark.parametrize("arena", [False, True])
def test_mix_equals_alone(arena):
    trace = _trace()
    budget = 3 * max(r.footprint() for r in trace)  # forces admission to wait for memory
    lau = CudaLauncher(n_streams=3, ws_bytes=64 << 20, keep_results=True, psf_arena_bytes=budget if arena else None)
    st = Scheduler(lau, budget, unit_lambdas=3).run(trace)
    torch.cuda.synchronize()
    assert st.summary()["completed"] == len(trace)
    assert st.peak_bytes <= budget
    assert st.launches < sum(-(-r.L // 3) for r in trace)  # some launches were shared
    for r in trace:
        assert torch.equal(lau.results[r.rid], _alone(r)), r.rid


def test_one_at_a_time_baseline_same_results():
    trace = _trace(n=8, seed=9)
    st, res = serve_one_at_a_time(trace, keep_results=True)
    assert st.summary()["completed"] == len(trace)
    for r in trace:
        assert torch.equal(res[r.rid], _alone(r))


# -------------------------------------------------------------- serving workload vs the oracle
# Requests shaped like the serving workload: sides N in {1024, ..., 16384} (grids 2048^2 to
# 32768^2), 1..31 wavelengths in [400, 700] nm, z in [10, 100] mm, 1 um pitch, Poisson arrivals
# at 200 requests/s, so that all of them are admitted and in flight together.  Wavelength counts
# of the large sides are capped so that every PSF of the trace fits on the device at once
# (4096: up to 12, 8192: up to 4, 16384: up to 2).
TOL_PSF = 1e-5
_C5_SIDES = [16384, 1024, 4096, 2048, 8192, 1024, 2048, 4096, 1024, 2048]
_C5_LMAX = {1024: 31, 2048: 31, 4096: 12, 8192: 4, 16384: 2}


def _c5_trace(seed=3005):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i, N in enumerate(_C5_SIDES):
        t += rng.exponential(1.0 / 200.0)
        L = int(rng.integers(1, _C5_LMAX[N] + 1))
        out.append(Req(rid=i, arrival_s=t, N=N, lambdas=rng.uniform(400e-9, 700e-9, L),
                       z=float(rng.uniform(10e-3, 100e-3)), seed=100000 + i))
    return out


def _rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_serving_mix_vs_oracle():
    """Each request's PSFs, computed in the continuous-batching mix (shared launches of
    several requests, three streams, admission under a budget that holds several large
    requests at once), against the FP64 oracle: in full for grids up to 8192^2 (two seeded
    wavelengths per request), on seeded rows for 16384^2 and 32768^2 (one seeded wavelength,
    the oracle's row-subset mode), relative L2 <= 1e-5 per wavelength.  Beside it, the mix
    equals the same request computed alone, bit for bit."""
    import oracle

    trace = _c5_trace()
    budget = 48 << 30
    lau = CudaLauncher(n_streams=3, ws_bytes=20 << 30, keep_results=True)
    st = Scheduler(lau, budget, unit_lambdas=8).run(trace)
    torch.cuda.synchronize()
    assert st.summary()["completed"] == len(trace)
    assert st.launches < sum(-(-r.L // 8) for r in trace)  # some launches were shared
    rng = np.random.default_rng(42)
    for r in trace:
        mix = lau.results[r.rid]
        assert torch.equal(mix, _alone(r)), r.rid
        h = heights_device(r.N, r.seed, "cuda").cpu().numpy()  # the heights the launcher used
        if r.P <= 8192:
            js = sorted(set(rng.choice(r.L, size=min(2, r.L), replace=False).tolist()))
            for j in js:
                ref = oracle.psf(h, r.dx, r.z, [float(r.lambdas[j])], n_index=r.n_index)[0]
                err = _rel_l2(mix[j].cpu().numpy(), ref)
                assert err <= TOL_PSF, (r.rid, r.N, j, err)
        else:
            j = int(rng.integers(0, r.L))
            rows = np.unique(np.concatenate([[0, r.P // 2 - 1, r.P // 2, r.P - 1], rng.integers(0, r.P, 4)]))
            ref = oracle.psf_rows(h, r.dx, r.z, float(r.lambdas[j]), rows, n_index=r.n_index)
            got = mix[j][torch.from_numpy(rows).cuda()].cpu().numpy()
            err = _rel_l2(got, ref)
            assert err <= TOL_PSF, (r.rid, r.N, j, err)
        del mix
        lau.results.pop(r.rid)
