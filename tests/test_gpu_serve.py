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
