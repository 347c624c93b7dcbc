"""GPU parity of the Monte Carlo prior weights (sec. 2.3, App. B) through the C ABI
(sr_noise_weights) against the FP64 oracle on the same random stream.

Both sides draw the same normals (Philox4x64-10, 24-bit uniforms, Box-Muller), so the comparison
is element by element, not statistical.  Tolerance, from the arithmetic: the GPU works in FP32
(normals to ~1e-7 relative, the K x K correlation and the starlet levels to ~1e-6 relative of the
coefficients they produce) and accumulates the moments in FP64, so a standard deviation over many
realisations carries ~1e-6 relative error; the bounds below are 2e-5 for the pooled per-scale W
and 1e-4 for the per-coefficient maps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL_SCALE, RTOL_MAP = 2e-5, 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _gpu(N, f, K, J, sigma, s1, n_real, seed, **kw):
    from paper_2402_08725_gb300.binding import noise_weights
    sg = torch.from_numpy(np.ascontiguousarray(sigma, dtype=np.float32)).cuda()
    sk = torch.from_numpy(np.ascontiguousarray(s1, dtype=np.float32)).cuda()
    Ws, Wm, tm = noise_weights(N, f, K, J, sg, sk, n_real, seed, **kw)
    return Ws, (Wm.cpu().numpy() if Wm is not None else None), tm


def _case(rng, N, f, K, E, mask=True):
    s1 = rng.random((K, K)) ** 2
    s1 /= s1.sum()
    sigma = rng.uniform(2.0, 9.0, (E, N, N))
    if mask:
        sigma[0, N // 3, N // 2] = np.inf
        sigma[:, 1, 1] = np.inf  # a pixel masked in every epoch: no noise there
    return sigma.astype(np.float32), s1.astype(np.float32)


def _compare(N, f, K, J, sigma, s1, n_real, seed):
    Ws_ref, Wm_ref = oracle.noise_weights(N, f, K, J, sigma.astype(np.float64), s1.astype(np.float64), n_real, seed)
    Ws, Wm, _ = _gpu(N, f, K, J, sigma, s1, n_real, seed)
    np.testing.assert_allclose(Ws, Ws_ref, rtol=RTOL_SCALE, atol=0)
    np.testing.assert_allclose(Wm, Wm_ref, rtol=RTOL_MAP, atol=RTOL_MAP * 1e-3 * float(np.max(Wm_ref)))
    return Ws, Wm


@pytest.mark.parametrize("N,f,K,J,E,n_real", [
    (12, 2, 9, 3, 3, 300),    # one tile, ragged columns, odd kernel
    (37, 1, 6, 3, 2, 50),     # odd grid, even kernel (origin K/2), kernel columns padded to 8
    (75, 2, 71, 4, 2, 6),     # 2 x 5 tiles with ragged edges, two kernel-row chunks
    (20, 3, 1, 4, 4, 100),    # delta PSF, f = 3
    (8, 1, 15, 3, 2, 200),    # PSF wider than the grid (K > F): taps outside read zero
    (16, 2, 5, 5, 1, 40),     # the deepest starlet of this grid: 2 * 2^(J-2) = 16 <= F - 1 = 31 (J = 6 needs 32)
])
def test_noise_weights_match_oracle(N, f, K, J, E, n_real):
    rng = np.random.default_rng(N * 100 + K)
    sigma, s1 = _case(rng, N, f, K, E)
    _compare(N, f, K, J, sigma, s1, n_real, seed=1000 + N)


def test_noise_weights_full_size_workload():
    """The measured workload: a 64 x 64 stamp field with 300 epochs, f = 2 (F = 128), the first
    epoch's 64 x 64 Moffat PSF, 4 starlet planes, 5000 realisations (App. B's count) in the
    launch configuration the benchmark times, every output against the oracle."""
    fd = syn.config3()
    Ws, Wm = _compare(fd.N, fd.f, fd.K, fd.J, fd.sigma, fd.s[0], 5000, seed=2402)
    # S_1^T smooths the noise with a PSF several pixels wide: the coarser scales carry more of it
    assert np.all(Ws > 0) and np.all(np.diff(Ws) > 0)


def test_noise_weights_deterministic_and_seeded():
    rng = np.random.default_rng(5)
    sigma, s1 = _case(rng, 24, 2, 11, 3)
    a = _gpu(24, 2, 11, 4, sigma, s1, 200, 9)
    b = _gpu(24, 2, 11, 4, sigma, s1, 200, 9)
    c = _gpu(24, 2, 11, 4, sigma, s1, 200, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_noise_weights_outputs_optional_and_timed():
    rng = np.random.default_rng(6)
    N, f, K, J = 32, 2, 15, 4
    sigma, s1 = _case(rng, N, f, K, 2)
    Ws_all, Wm_all, _ = _gpu(N, f, K, J, sigma, s1, 64, 3)
    Ws, Wm, tm = _gpu(N, f, K, J, sigma, s1, 64, 3, want_map=False, timing=True)
    assert Wm is None and np.array_equal(Ws, Ws_all)
    assert tm["corr_ms"] > 0 and tm["starlet_ms"] > 0 and tm["draw_ms"] > 0
    nb = -(-64 // tm["batch"])
    assert tm["launches"] == 1 + nb * (2 + 2 * (J - 1)) + 1


def test_noise_weights_rejects_bad_input():
    from paper_2402_08725_gb300 import _native as nat
    rng = np.random.default_rng(7)
    sigma, s1 = _case(rng, 16, 2, 5, 2, mask=False)
    bad = sigma.copy()
    bad[1, 3, 3] = np.nan
    with pytest.raises(RuntimeError, match="SR_ERR_NONFINITE"):
        _gpu(16, 2, 5, 3, bad, s1, 10, 0)
    bad = sigma.copy()
    bad[0, 0, 0] = 0.0
    with pytest.raises(RuntimeError, match="SR_ERR_NONFINITE"):
        _gpu(16, 2, 5, 3, bad, s1, 10, 0)
    with pytest.raises(RuntimeError, match="SR_ERR_SHAPE"):
        _gpu(16, 2, 5, 7, sigma, s1, 10, 0)  # 2 * 2^5 > F - 1
    with pytest.raises(RuntimeError, match="SR_ERR_SHAPE"):
        _gpu(16, 2, 5, 3, sigma, s1, 1, 0)
    # the error leaves the context usable
    Ws, _, _ = _gpu(16, 2, 5, 3, sigma, s1, 10, 0)
    assert np.all(np.isfinite(Ws)) and nat.load() is not None
