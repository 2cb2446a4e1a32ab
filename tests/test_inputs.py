"""Host checks of the seeded input generators (no method arithmetic lives there)."""
import numpy as np
from scipy import ndimage

from paper_2505_22313_b300 import inputs


def test_flat_top_target_is_an_equal_intensity_8x8_lattice():
    P, N = 512, 256
    T = inputs.flat_top_target(P, N, 3)
    assert T.shape == (3, P, P) and T.dtype == np.float32
    for j in range(3):
        assert abs(float(T[j].astype(np.float64).sum()) - N * N) <= 1e-5 * N * N
        assert np.array_equal(T[j], T[0])
    vals = np.unique(T[0])
    assert vals.size == 2 and vals[0] == 0.0  # flat-top: one intensity level
    lab, n = ndimage.label(T[0] > 0)
    assert n == 64
    sizes = ndimage.sum(np.ones_like(lab), lab, index=np.arange(1, n + 1))
    assert np.all(sizes == sizes[0])  # equal spots
    cy, cx = np.array(ndimage.center_of_mass(T[0] > 0))
    assert abs(cy - P / 2) < 1.0 and abs(cx - P / 2) < 1.0  # centred on the optical axis
