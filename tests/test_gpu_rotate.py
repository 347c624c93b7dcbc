"""GPU parity of rotated frames (sec. 5 rotations between frames: epoch i's frame turned by
theta_i about the grid centre, h read bilinearly with zero outside, sources at
u0 + f (R c_k + delta_i)) against the FP64 oracle, through the C ABI, with and without the
extended channel moving with the shifts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import check_deconv  # noqa: E402
import oracle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _field(seed, E, N, f, K, M, J, span=0.6):
    fd = syn.small_deconv(seed=seed, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.1)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    rng = np.random.default_rng(seed + 7)
    dl = rng.uniform(-span, span, size=(E, 2))
    fd.params = syn.pack_deconv(h, a, c, dl, gm)
    theta = rng.uniform(-np.pi, np.pi, size=E)
    return fd, theta


def _check(fd, theta, shifted, conv_mode="auto"):
    from paper_2402_08725_gb300.binding import Problem
    prob = Problem.from_field(fd, conv_mode=conv_mode)
    prob.set_translate_h(shifted)
    prob.set_rotations(theta)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(p)
    g = grad.cpu().numpy()
    prob.close()
    return check_deconv(fd, loss, g, shifted=shifted, theta=theta)


CASES = [
    (3, 24, 2, 15, 2, 3),
    (2, 20, 3, 17, 1, 3),
    (2, 16, 1, 9, 2, 3),
    (3, 37, 2, 12, 0, 3),
    (2, 70, 3, 30, 2, 5),
    (5, 64, 2, 64, 3, 4),
]


@pytest.mark.parametrize("E,N,f,K,M,J", CASES)
@pytest.mark.parametrize("shifted", [False, True])
def test_rotated_frames_match_oracle(E, N, f, K, M, J, shifted):
    fd, theta = _field(1700 + N + K, E, N, f, K, M, J)
    r = _check(fd, theta, shifted)
    print("rotated", E, N, f, K, M, shifted, r)


def test_quarter_turns_and_masked_pixels():
    fd, _ = _field(1800, E=4, N=28, f=2, K=13, M=2, J=3, span=0.9)
    fd.sigma[2, 4:10, 6:18] = np.inf
    theta = np.array([0.0, np.pi / 2, np.pi, -np.pi / 2]) + 1e-3
    _check(fd, theta, True, conv_mode="direct")


def test_zero_angles_leave_the_loss_unchanged():
    """theta = 0 without the moved channel reads h at the pixel itself: the same loss bit for
    bit as the unrotated evaluation."""
    from paper_2402_08725_gb300.binding import Problem
    fd, _ = _field(1900, E=3, N=32, f=2, K=15, M=2, J=3)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    prob = Problem.from_field(fd, conv_mode="direct")
    l0, g0 = prob.loss_and_grad(p)
    prob.set_rotations(np.zeros(fd.E))
    l1, g1 = prob.loss_and_grad(p)
    assert l1 == l0
    assert torch.allclose(g1, g0, rtol=1e-5, atol=1e-6 * float(g0.abs().max()))
    prob.close()


def test_new_angles_take_effect_without_a_new_plan():
    from paper_2402_08725_gb300.binding import Problem
    fd, theta = _field(2000, E=3, N=24, f=2, K=15, M=2, J=3)
    prob = Problem.from_field(fd)
    prob.set_rotations(theta)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    prob.loss_and_grad(p)
    theta2 = theta[::-1] + 0.3
    prob.set_rotations(theta2)
    loss, grad = prob.loss_and_grad(p)
    check_deconv(fd, loss, grad.cpu().numpy(), theta=theta2)
    prob.close()


@pytest.mark.parametrize("mode", ["fft", "plain"])
def test_rotations_need_the_direct_form(mode):
    from paper_2402_08725_gb300.binding import Problem
    fd, theta = _field(2100, E=2, N=24, f=2, K=15, M=1, J=3)
    prob = Problem.from_field(fd, conv_mode=mode)
    with pytest.raises(RuntimeError):
        prob.set_rotations(theta)
    prob.close()


def test_rotated_fields_in_a_batch_equal_single_and_toggle_needs_recreate():
    from paper_2402_08725_gb300.binding import Batch, Problem
    f0, t0 = _field(2200, E=3, N=24, f=2, K=15, M=1, J=3)
    f1 = syn.small_deconv(seed=2201, E=2, N=32, f=2, K=17, M=2, J=3)
    f2, t2 = _field(2202, E=4, N=20, f=3, K=13, M=2, J=3)
    fields = [f0, f1, f2]
    probs = [Problem.from_field(fd) for fd in fields]
    probs[0].set_rotations(t0)
    probs[2].set_rotations(t2)
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
    check_deconv(f0, losses[0].item(), grad[:f0.n_params].cpu().numpy(), theta=t0)
    probs[1].set_rotations(np.zeros(f1.E))
    with pytest.raises(RuntimeError):
        batch.loss_and_grad(P, losses=losses)
    batch.close()
    for pr in probs:
        pr.close()


def test_rotation_angles_are_checked():
    from paper_2402_08725_gb300.binding import Problem
    fd, theta = _field(2300, E=2, N=16, f=2, K=9, M=1, J=3)
    prob = Problem.from_field(fd)
    bad = theta.copy()
    bad[1] = np.nan
    with pytest.raises(RuntimeError):
        prob.set_rotations(bad)
    with pytest.raises(ValueError):
        prob.set_rotations(theta[:1])
    prob.close()
    assert oracle is not None
