"""Host-logic checks of the seeded generators (CPU): the per-epoch host blur conserves flux
(up to what spills off the stamp), widens with the seeing, and leaves the default draw unchanged."""
import numpy as np

from paper_2402_08725_gb300 import synthetic as syn


def _moment2(img):
    n = img.shape[0]
    y, x = np.mgrid[0:n, 0:n] - (n - 1) / 2.0
    return float(np.sum(img * (x * x + y * y)) / np.sum(img))


def test_blurred_host_conserves_flux_and_widens_with_seeing():
    host = [{"flux": 3e4, "n": 4.0, "re": 4.0}, {"flux": 5e4, "n": 1.0, "re": 12.0, "q": 0.6}]
    fw = np.array([2.0, 3.0, 4.5])
    st = syn.blurred_host_stack(host, 64, 2, fw, np.array([3.0, 3.0, 3.0]))
    sharp = syn.blurred_host_stack(host, 64, 2, np.array([1e-3]), np.array([3.0]))[0]
    assert abs(sharp.sum() - 8e4) <= 2e-3 * 8e4
    for img in st:
        assert 0.97 * 8e4 <= img.sum() <= 8e4 * (1 + 1e-6)
    m = [_moment2(img) for img in st]
    assert m[0] < m[1] < m[2]
    assert _moment2(sharp) < m[0]


def test_default_host_draw_is_unchanged_by_the_option():
    a = syn.config4_field(3, 48, 20, 4)
    b = syn.config4_field(3, 48, 20, 4, host_blur="mean")
    np.testing.assert_array_equal(a.d, b.d)
    c = syn.config4_field(3, 48, 20, 4, host_blur="epoch")
    np.testing.assert_array_equal(a.params, c.params)
    assert not np.array_equal(a.d, c.d)
