"""The kernels' fault word: a bounded wait that runs out is reported to the host through
doe_fault_status and the context stays usable (no trap, no hang, no fault).  The wait is on an
mbarrier that announces a copy nobody issues; its poll bound is small, so it gives up at once."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_22313_b300 import _lib as L
from paper_2505_22313_b300 import api, inputs
from paper_2505_22313_b300.api import Geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2505_22313_b300 import build

    build.build()
    assert torch.cuda.is_available()
    api.init()


def test_wait_timeout_sets_fault_bit_and_context_stays_usable():
    api.fault_status()  # clear
    api.check_wait_timeout(1 << 10)
    assert api.fault_status() & L.DOE_FAULT_WAIT_TIMEOUT
    assert api.fault_status() == 0  # read and cleared
    # the context still runs the path and its results still match the oracle
    N, dx, z, lam = 64, 1e-6, 1e-3, 550e-9
    h = inputs.heights(N, 4242)
    I = api.psf(torch.from_numpy(h).cuda(), Geometry.make(N, dx, z, [lam])).cpu().numpy()
    ref = oracle.psf(h, dx, z, [lam])
    assert float(np.linalg.norm((I - ref).ravel()) / np.linalg.norm(ref.ravel())) < 1e-5
    assert api.fault_status() == 0
