"""End-to-end extraction through the library's captured optimiser steps (sec. 2.4, sec. 3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_08725_gb300 import metrics as mt  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def test_recovery_of_point_sources_noiseless_on_gpu():
    """The oracle's noiseless recovery pin run through sr_step: data made by the oracle's model,
    AdaBelief on (a, c) from a * 1.2 and c + 0.3 px, 1500 steps (lr / 10 after 1000) recovers the
    amplitudes to 1e-3 relative and the positions to 1e-3 px."""
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    fd = syn.small_deconv(seed=21, E=3, N=14, f=2, K=9, M=2, J=3, lam=0.0)
    E, N, f, K, M, J = fd.E, fd.N, fd.f, fd.K, fd.M, fd.J
    truth = fd.params.astype(np.float64)
    d = oracle.deconv_model(E, N, f, K, M, fd.s, truth)
    h, a, c, dl, gm = syn.unpack_deconv(truth, E, N, f, M)
    start = syn.pack_deconv(h, a * 1.2, c + 0.3, dl, gm)
    p = Problem("deconv", E, N, f, K, M, J, 0.0)
    p.set_data(d.astype(np.float32))
    p.set_noise(np.full((E, N, N), 3.0, dtype=np.float32))
    p.set_psfs(fd.s)
    p.set_weights(fd.W)
    P = torch.from_numpy(np.ascontiguousarray(start, dtype=np.float32)).cuda()
    lr = (0.0, 0.02 * float(np.abs(a).mean()), 0.01, 0.0, 0.0)
    p.step(P, 1000, optim_cfg("adabelief", lr=lr))
    p.step(P, 500, optim_cfg("adabelief", lr=tuple(x * 0.1 for x in lr)))
    _, a_r, c_r, _, _ = syn.unpack_deconv(P.cpu().numpy().astype(np.float64), E, N, f, M)
    np.testing.assert_allclose(a_r, a, rtol=1e-3)
    np.testing.assert_allclose(c_r, c, atol=1e-3)
    assert mt.a_photo(a, a_r) == pytest.approx(0.0, abs=1e-3) and mt.p_astro(c, c_r) < 1e-3
    p.close()


def test_extraction_of_a_noisy_point_source_field():
    """60 epochs of 32 x 32 with one point source on the sky: 600 steps reach chi^2 ~ half the
    pixel count, the photometry is unbiased within 1 % and scatters by about the noise (the
    metrics of sec. 3), and the position is found to 0.05 px from a 0.2 px catalogue error."""
    from paper_2402_08725_gb300.extract import extract
    fd = syn.point_source_field(6, E=60, N=32, M=1)
    _, a_t, c_t, _, _ = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    c0 = c_t + np.random.default_rng(1).normal(0.0, 0.2, c_t.shape)
    res = extract(fd, c0, n_steps=600, lambda_pts=0.0)
    L = res["losses"]
    npix = fd.E * fd.N * fd.N
    assert np.all(np.isfinite(L)) and abs(L[-1] / (0.5 * npix) - 1.0) < 0.05
    assert abs(mt.a_photo(a_t, res["a"])) < 0.01 and mt.p_photo(a_t, res["a"]) < 0.03
    assert np.max(np.abs(res["c"] - c_t)) < 0.05


def test_extraction_refines_lambda_pts_by_app_c():
    """The App. C rounds: lambda_pts starts at 0.5 lambda and each round takes the estimate."""
    from paper_2402_08725_gb300.extract import extract
    fd = syn.point_source_field(8, E=20, N=32, M=2)
    _, a_t, c_t, _, _ = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    res = extract(fd, c_t, n_steps=300, lambda_pts="app_c", rounds=3)
    assert len(res["lambda_pts"]) == 3 and res["lambda_pts"][0] == 0.5 * fd.lam
    assert all(np.isfinite(v) and v >= 0.0 for v in res["lambda_pts"])
    assert np.all(np.isfinite(res["losses"]))


def test_extraction_of_a_lensed_quasar_on_its_host():
    """Config 3 with the host drawn through each epoch's seeing (so that one h fits every epoch):
    the four images' light curves and positions come out of 200 steps with the point-source
    prior at its App. C estimate, next to the ring arc and the lens galaxy: chi^2 within 10 % of
    half the pixel count, photometry within 15 % with a scatter below 10 %, positions to 0.05 px."""
    from paper_2402_08725_gb300.extract import extract
    fd = syn.config3(host_blur="epoch")
    _, a_t, c_t, _, _ = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    c0 = c_t + np.random.default_rng(1).normal(0.0, 0.2, c_t.shape)
    res = extract(fd, c0, n_steps=200, lambda_pts="app_c")
    npix = fd.E * fd.N * fd.N
    assert abs(res["losses"][-1] / (0.5 * npix) - 1.0) < 0.1
    bright = a_t >= 0.1 * a_t.max(axis=0, keepdims=True)
    assert abs(mt.a_photo(a_t, res["a"], bright)) < 0.15
    assert mt.p_photo(a_t, res["a"], bright) < 0.10
    assert mt.p_astro(c_t, res["c"]) < 0.05
