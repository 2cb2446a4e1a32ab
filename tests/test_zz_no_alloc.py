"""doe_psf_noalloc: the PSF entry point for callers that cannot allocate device memory.

Such callers (a plugin that receives only its input and output buffers from a host
application owning the device-memory budget, or a loop that must never call cudaMalloc)
cannot provide doe_psf's workspace; this entry point uses a static scratch array inside the
library instead.  Checked through the C ABI against doe_psf on two calls in a row (the second
with different heights, so stale scratch contents would show), then on a sequence in which
the scratch layout moves (a mixed-radix grid after a larger power-of-two one, a smaller grid
after a larger one, a call with an incident field), plus the size limit.  This file sorts last
so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_22313_b300 import _lib as L
from paper_2505_22313_b300 import api, build, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, as for every PSF test


@pytest.fixture(scope="module")
def lib():
    build.build()
    assert torch.cuda.is_available()
    return L.load()


def _call(lib, g, h, out, e_in=None):
    gc = g.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.doe_psf_noalloc(ctypes.byref(gc), ctypes.c_void_p(h.data_ptr()),
                               None if e_in is None else ctypes.c_void_p(e_in.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), stream)


def _check(lib, g, h, e_in=None):
    assert api.workspace_bytes(g, L.DOE_OP_PSF) <= L.DOE_NOALLOC_SCRATCH_BYTES
    out = torch.full((g.L, g.P, g.P), float("nan"), dtype=torch.float32, device="cuda")
    assert _call(lib, g, h, out, e_in) == L.DOE_OK
    ref = api.psf(h, g, e_in=e_in)
    torch.cuda.synchronize()
    err = (torch.linalg.vector_norm((out - ref).double()) / torch.linalg.vector_norm(ref.double())).item()
    assert np.isfinite(err) and err <= TOL, err


def test_psf_noalloc_matches_psf_on_two_calls(lib):
    N, dx, z = 256, 2e-6, 20e-3
    g = Geometry.make(N, dx, z, [450e-9, 550e-9, 650e-9])
    for seed in (1001, 1077):
        _check(lib, g, torch.from_numpy(inputs.heights(N, seed)).cuda())


def test_psf_noalloc_sequence_with_moving_layouts(lib):
    # a large power-of-two grid whose workspace nearly fills the scratch, then layouts that
    # place their buffers differently: a mixed-radix grid (360 = 2^3 3^2 5, per-call twiddle
    # tables at the end of its workspace), a non-power-of-two 180 grid, a smaller power-of-two
    # grid, and one call with an incident field array
    rng = np.random.default_rng(11)
    big = Geometry.make(1024, 1e-6, 8e-3, [550e-9], pad=2)  # 2048^2 grid, ~24 MiB of the 32 MiB scratch
    assert api.workspace_bytes(big, L.DOE_OP_PSF) > 16 << 20
    seq = [(big, 1024), (Geometry.make(360, 1e-6, 2e-3, [450e-9, 633e-9]), 360),
           (Geometry.make(180, 1e-6, 1e-3, [550e-9]), 180), (Geometry.make(128, 1e-6, 2e-3, [532e-9]), 128)]
    for g, N in seq:
        _check(lib, g, torch.from_numpy(inputs.heights(N, 1000 + N)).cuda())
    N = 96
    g = Geometry.make(N, 1e-6, 1e-3, [500e-9, 600e-9])
    e_in = torch.from_numpy((rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64))
    _check(lib, g, torch.from_numpy(inputs.heights(N, 1096)).cuda(), e_in.cuda())


def test_psf_noalloc_rejects_oversize(lib):
    # the smallest kind of geometry past the limit: 1024^2 DOE, 2x padding, one wavelength at
    # a short distance (band limit inactive), so the [2048][2048] complex field alone is
    # 32 MiB.  The buffers are allocated at full size, so a broken size check would compute a
    # result instead of touching memory out of bounds.
    g = Geometry.make(1024, 1e-6, 1e-3, [550e-9])
    assert api.workspace_bytes(g, L.DOE_OP_PSF) > L.DOE_NOALLOC_SCRATCH_BYTES
    h = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, g.P, g.P), dtype=torch.float32, device="cuda")
    assert _call(lib, g, h, out) == L.DOE_ESCRATCH
