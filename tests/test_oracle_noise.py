"""Pins for the oracle's noise propagation (sec. 2.3, App. B): the counter-based
generator, the Gaussian draws and the Monte Carlo weight maps W.

Each pin comes from outside the oracle: NumPy's own Philox4x64-10 bit generator,
the moments and quantiles of the standard normal law, the published white-noise
standard deviations of the B3 starlet scales, and the exact variance of the
linear map  z -> Phi S_1^T (C^)^-1/2 z  built column by column with scipy."""
import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

import oracle

B3 = np.array([1, 4, 6, 4, 1], dtype=np.float64) / 16.0


@pytest.mark.parametrize("key", [(12345, 0), (0, 0), (2**64 - 1, 7)])
def test_philox_matches_numpy_bit_generator(key):
    """NumPy's Philox increments the counter before each block, so its words
    4(c-1) .. 4c-1 are the block for counter c."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
    raw = [int(w) for w in bg.random_raw(12)]
    for c in (1, 2, 3):
        assert oracle.philox4x64([c, 0, 0, 0], key) == raw[4 * (c - 1): 4 * c]


def test_philox_high_counter_words():
    """A counter with all four words set, against NumPy started one block below it."""
    ctr = [5, 2**63 + 3, 11, 2**40]
    key = (99, 2**33)
    start = np.array([ctr[0] - 1, ctr[1], ctr[2], ctr[3]], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    assert oracle.philox4x64(ctr, key) == [int(w) for w in bg.random_raw(4)]


def test_normal_draws_have_standard_moments_and_quantiles():
    n = 200_000
    z = np.array([oracle.normal(2024, k) for k in range(n)])
    se = 1.0 / np.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0) * se
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0) * se  # Var(z^4) = 105 - 9
    for q, p in ((0.0, 0.5), (1.0, 0.841344746), (-1.96, 0.024997895)):
        frac = np.mean(z < q)
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p)) * se
    assert np.all(np.isfinite(z)) and np.max(np.abs(z)) < 6.5


def test_normal_streams_depend_on_seed_and_index():
    a = [oracle.normal(1, k) for k in range(64)]
    assert a == [oracle.normal(1, k) for k in range(64)]
    b = [oracle.normal(2, k) for k in range(64)]
    assert not np.allclose(a, b)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.5
    assert len(set(a)) == 64


# published standard deviations of the B3 starlet detail scales under unit white noise
# (tests/golden/starlet_b3_white_noise.txt, with its citation)
_GOLDEN = __file__.rsplit("/", 1)[0] + "/golden/starlet_b3_white_noise.txt"
STARLET_WHITE_NOISE = [float(l.split()[1]) for l in open(_GOLDEN) if not l.startswith("#")]


def test_weights_white_noise_match_published_starlet_norms():
    """Delta PSF, four epochs of sigma 2 (co-added sigma 1) plus one masked epoch:
    away from the borders W_j is the white-noise norm of starlet scale j."""
    N, f, K, J = 32, 2, 1, 5
    sigma = np.full((5, N, N), 2.0)
    sigma[4] = np.inf
    _, W = oracle.noise_weights(N, f, K, J, sigma, np.ones((1, 1)), n_real=200, seed=3)
    assert W.shape == (J - 1, f * N, f * N)
    for j in range(3):
        r = 2 * (2 ** (j + 1) - 1)  # half-width of the cascade down to scale j
        inner = W[j, r:-r, r:-r]
        assert abs(np.sqrt(np.mean(inner ** 2)) / STARLET_WHITE_NOISE[j] - 1.0) < 0.03


def _starlet_details(h, J):
    out, c = [], h
    for j in range(J - 1):
        k = np.zeros(4 * (1 << j) + 1)
        k[:: 1 << j] = B3
        cn = scipy.ndimage.correlate1d(c, k, axis=1, mode="mirror")
        cn = scipy.ndimage.correlate1d(cn, k, axis=0, mode="mirror")
        out.append(c - cn)
        c = cn
    return np.array(out)


def _exact_std(isig, s1, J, flip=False):
    """Per-coefficient std of Phi S^T diag(isig) z for z ~ N(0, I), summed over columns."""
    F = isig.shape[0]
    var = np.zeros((J - 1, F, F))
    k = s1[::-1, ::-1] if flip else s1
    for u in range(F * F):
        e = np.zeros((F, F))
        e.flat[u] = isig.flat[u]
        var += _starlet_details(scipy.signal.correlate2d(e, k, mode="same"), J) ** 2
    return np.sqrt(var)


def test_weights_match_exact_variance_of_the_linear_map():
    """Asymmetric PSF, per-pixel noise spread over a decade, one masked pixel: the
    Monte Carlo W against the exact std of the linear map."""
    rng = np.random.default_rng(8)
    N, f, K, J, E = 6, 2, 5, 3, 3
    s1 = rng.random((K, K)) ** 3
    s1 /= s1.sum()
    sigma = np.exp(rng.normal(0.0, 1.0, (E, N, N)))
    sigma[1, 2, 3] = np.inf
    isig = np.sqrt(np.sum(np.where(np.isfinite(sigma), 1.0 / sigma ** 2, 0.0), axis=0))
    isig = np.kron(isig, np.ones((f, f)))  # C^: the noise map replicated on the fine grid
    exact = _exact_std(isig, s1, J)
    Ws, W = oracle.noise_weights(N, f, K, J, sigma, s1, n_real=20000, seed=11)
    rel = W / exact - 1.0
    assert np.max(np.abs(rel)) < 0.03  # 1/sqrt(2n) = 0.5 % per value
    assert abs(np.mean(rel)) < 0.005
    # pooled over a scale (zero-mean coefficients): the mean of the exact per-pixel variances
    pooled = np.sqrt(np.mean(exact.reshape(J - 1, -1) ** 2, axis=1))
    np.testing.assert_allclose(Ws, pooled, rtol=0.01)
    # the pin separates the right operator from its mirror image and from C instead of C^-1
    assert np.max(np.abs(_exact_std(isig, s1, J, flip=True) / exact - 1.0)) > 0.1
    assert np.max(np.abs(np.log(_exact_std(1.0 / isig, s1, J) / exact))) > 1.0


def test_pooled_weights_follow_the_co_added_noise_level():
    """Scaling every sigma by t scales W by 1/t; E epochs of equal sigma weigh like one epoch of
    sigma / sqrt(E); the same stream gives the same numbers."""
    rng = np.random.default_rng(4)
    N, f, K, J = 8, 2, 3, 3
    s1 = rng.random((K, K))
    sig = rng.uniform(1.0, 3.0, (1, N, N))
    Ws1, Wm1 = oracle.noise_weights(N, f, K, J, sig, s1, n_real=50, seed=5)
    Ws2, Wm2 = oracle.noise_weights(N, f, K, J, 2.5 * sig, s1, n_real=50, seed=5)
    np.testing.assert_allclose(Ws2, Ws1 / 2.5, rtol=1e-12)
    np.testing.assert_allclose(Wm2, Wm1 / 2.5, rtol=1e-12)
    Ws4, _ = oracle.noise_weights(N, f, K, J, np.repeat(sig * 2.0, 4, axis=0), s1, n_real=50, seed=5)
    np.testing.assert_allclose(Ws4, Ws1, rtol=1e-12)
    Ws5, _ = oracle.noise_weights(N, f, K, J, sig, s1, n_real=50, seed=6)
    assert np.all(np.abs(Ws5 / Ws1 - 1.0) > 1e-6)


def test_weights_reject_bad_shapes():
    with pytest.raises(Exception):
        oracle.noise_weights(4, 1, 3, 4, np.ones((1, 4, 4)), np.ones((3, 3)), n_real=10, seed=0)
    with pytest.raises(Exception):
        oracle.noise_weights(8, 1, 3, 3, np.ones((1, 8, 8)), np.ones((3, 3)), n_real=1, seed=0)
