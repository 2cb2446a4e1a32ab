"""doe_psf_noalloc: the PSF entry point for callers that cannot allocate device memory.

Such callers (a plugin that receives only its input and output buffers from a host
application owning the device-memory budget, or a loop that must never call cudaMalloc)
cannot provide doe_psf's workspace; this entry point uses a static scratch array inside the
library instead.  Checked through the C ABI against doe_psf on two calls in a row (the second
with different heights, so stale scratch contents would show), plus the size limit.  This
file sorts last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_22313_b300 import _lib as L
from paper_2505_22313_b300 import api, build, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available()
    return L.load()


def _call(lib, g, h, out):
    gc = g.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.doe_psf_noalloc(ctypes.byref(gc), ctypes.c_void_p(h.data_ptr()), None,
                               ctypes.c_void_p(out.data_ptr()), stream)


def test_psf_noalloc_matches_psf_on_two_calls(lib):
    N, dx, z = 256, 2e-6, 20e-3
    g = Geometry.make(N, dx, z, [450e-9, 550e-9, 650e-9])
    assert api.workspace_bytes(g, L.DOE_OP_PSF) <= L.DOE_NOALLOC_SCRATCH_BYTES
    for seed in (1001, 1077):
        h = torch.from_numpy(inputs.heights(N, seed)).cuda()
        out = torch.full((g.L, g.P, g.P), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, g, h, out) == L.DOE_OK
        ref = api.psf(h, g)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm((out - ref).double()) / torch.linalg.vector_norm(ref.double())).item()
        assert np.isfinite(err) and err <= 1e-5, err


def test_psf_noalloc_rejects_oversize(lib):
    g = Geometry.make(4096, 1e-6, 50e-3, [550e-9])
    assert api.workspace_bytes(g, L.DOE_OP_PSF) > L.DOE_NOALLOC_SCRATCH_BYTES
    h = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    out = torch.zeros((4,), dtype=torch.float32, device="cuda")
    assert _call(lib, g, h, out) == L.DOE_ESCRATCH
