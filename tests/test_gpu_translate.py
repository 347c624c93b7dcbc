"""GPU parity of the moved extended channel (sec. 5: h follows each epoch's frame shift
f * delta_i, bilinear with zero outside the grid) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import check_deconv  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _field(seed, E, N, f, K, M, J, span):
    """A small field whose epoch shifts span +-span data pixels (several fine pixels at f > 1,
    negative and positive, never a whole fine pixel where the interpolant has its kinks)."""
    fd = syn.small_deconv(seed=seed, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.3)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    rng = np.random.default_rng(seed + 1)
    dl = rng.uniform(-span, span, size=(E, 2))
    frac = f * dl - np.floor(f * dl)
    dl += ((frac < 0.02) * 0.05 - (frac > 0.98) * 0.05) / f
    fd.params = syn.pack_deconv(h, a, c, dl, gm)
    return fd


def _run(fd, conv_mode="auto", translate=True):
    from paper_2402_08725_gb300.binding import Problem
    prob = Problem.from_field(fd, conv_mode=conv_mode)
    prob.set_translate_h(translate)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(p)
    g = grad.cpu().numpy()
    prob.close()
    return loss, g


# (E, N, f, K, M, J, span): ragged tiles, f = 1, 2, 3, no sources, shifts up to 2.5 data pixels
CASES = [
    (3, 24, 2, 15, 2, 3, 0.6),
    (2, 20, 3, 17, 1, 3, 1.4),
    (2, 16, 1, 9, 2, 3, 2.5),
    (3, 37, 2, 12, 0, 3, 1.0),
    (2, 70, 3, 30, 2, 5, 0.4),
    (5, 64, 2, 64, 3, 4, 2.0),
]


@pytest.mark.parametrize("E,N,f,K,M,J,span", CASES)
@pytest.mark.parametrize("mode", ["auto", "direct"])
def test_moved_channel_matches_oracle(E, N, f, K, M, J, span, mode):
    fd = _field(1200 + N + K, E, N, f, K, M, J, span)
    loss, g = _run(fd, conv_mode=mode)
    r = check_deconv(fd, loss, g, shifted=True)
    print("moved channel", E, N, f, K, M, mode, r)


def test_moved_channel_masked_pixels_and_backgrounds():
    fd = _field(1300, E=3, N=28, f=2, K=13, M=2, J=3, span=1.2)
    fd.sigma[1, 3:9, 10:20] = np.inf
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    fd.params = syn.pack_deconv(h, a, c, dl, np.array([-0.2, 0.1, 0.35]))
    loss, g = _run(fd)
    check_deconv(fd, loss, g, shifted=True)


def test_zero_shifts_leave_the_loss_unchanged():
    """At delta = 0 the moved channel is h itself: the same loss bit for bit, and the h block
    within FP32 rounding of the unmoved evaluation (the epochs are summed in another order)."""
    fd = _field(1400, E=4, N=32, f=2, K=15, M=2, J=3, span=0.5)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    fd.params = syn.pack_deconv(h, a, c, np.zeros_like(dl), gm)
    l1, g1 = _run(fd, conv_mode="direct", translate=True)
    l0, g0 = _run(fd, conv_mode="direct", translate=False)
    assert l1 == l0
    F = fd.F
    assert np.linalg.norm(g1[:F * F] - g0[:F * F]) <= 1e-6 * np.linalg.norm(g0[:F * F])
    check_deconv(fd, l1, g1, shifted=True)


@pytest.mark.parametrize("mode", ["fft", "plain"])
def test_moved_channel_needs_the_direct_form(mode):
    from paper_2402_08725_gb300.binding import Problem
    fd = _field(1500, E=2, N=24, f=2, K=15, M=1, J=3, span=0.5)
    prob = Problem.from_field(fd, conv_mode=mode)
    with pytest.raises(RuntimeError):
        prob.set_translate_h(True)
    prob.close()


def test_moved_channel_in_a_batch_equals_single_and_toggle_needs_recreate():
    from paper_2402_08725_gb300.binding import Batch, Problem
    fields = [_field(1600, E=3, N=24, f=2, K=15, M=1, J=3, span=0.8),
              syn.small_deconv(seed=1601, E=2, N=32, f=2, K=17, M=2, J=3),
              _field(1602, E=4, N=20, f=3, K=13, M=2, J=3, span=1.1)]
    probs = [Problem.from_field(fd) for fd in fields]
    probs[0].set_translate_h(True)
    probs[2].set_translate_h(True)
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    total, grad = batch.loss_and_grad(P, losses=losses)
    for i, (fd, pr) in enumerate(zip(fields, probs)):
        l_i, g_i = pr.loss_and_grad(torch.from_numpy(fd.params).cuda())
        o = batch.offsets[i]
        assert losses[i].item() == l_i
        assert torch.equal(grad[o:o + fd.n_params], g_i)
        check_deconv(fd, l_i, g_i.cpu().numpy(), shifted=i != 1)
    probs[1].set_translate_h(True)
    with pytest.raises(RuntimeError):
        batch.loss_and_grad(P, losses=losses)
    batch.close()
    for pr in probs:
        pr.close()
