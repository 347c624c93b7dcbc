"""GPU parity of per-coefficient prior weights W_j(u) (sr_set_weight_map; the noise of sec. 2.3 and
App. B propagated to a map per scale) against the FP64 oracle with the same map: the
deconvolution in each form, the PSF fit, the point-source prior, batches, and clearing the map."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import check_deconv, check_psf, loss_errors, rel_l2, LOSS_RTOL, GRAD_RTOL  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _map(rng, W, F):
    W = np.asarray(W, dtype=np.float64)
    return (rng.uniform(0.3, 3.0, (W.size, F, F)) * W[:, None, None]).astype(np.float32)


@pytest.mark.parametrize("mode", ["direct", "fft", "plain"])
@pytest.mark.parametrize("E,N,f,K,M,J", [(3, 24, 2, 15, 2, 3), (2, 40, 2, 21, 1, 4), (2, 20, 3, 17, 1, 3)])
def test_deconvolution_with_a_weight_map_matches_oracle(E, N, f, K, M, J, mode):
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=2400 + N + K, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.5)
    Wm = _map(np.random.default_rng(N), fd.W, fd.F)
    prob = Problem.from_field(fd, conv_mode=mode)
    prob.set_weight_map(Wm)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(p)
    ref = copy.copy(fd)
    ref.W = Wm
    check_deconv(ref, loss, grad.cpu().numpy())
    # cleared: the per-scale weights again, bit for bit as a problem that never had a map
    prob.set_weight_map(None)
    l0, g0 = prob.loss_and_grad(p)
    prob.close()
    fresh = Problem.from_field(fd, conv_mode=mode)
    l1, g1 = fresh.loss_and_grad(p)
    fresh.close()
    assert l0 == l1 and torch.equal(g0, g1)


def test_psf_fit_with_a_weight_map_matches_oracle():
    from paper_2402_08725_gb300.binding import Problem
    pb = syn.small_psf(2500, S=3, N=16, f=2, J=3, lam=1.0)
    Wm = _map(np.random.default_rng(3), pb.W, pb.f * pb.N)
    prob = Problem.from_psf(pb)
    prob.set_weight_map(torch.from_numpy(Wm).cuda())   # from device memory
    P = torch.from_numpy(np.ascontiguousarray(pb.params, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(P)
    prob.close()
    ref = copy.copy(pb)
    ref.W = Wm
    check_psf(ref, loss, grad.cpu().numpy())


def test_point_source_prior_with_a_weight_map():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=2600, E=3, N=24, f=2, K=15, M=2, J=3, lam=1.2)
    Wm = _map(np.random.default_rng(5), fd.W, fd.F)
    prob = Problem.from_field(fd, conv_mode="direct")
    prob.set_weight_map(Wm)
    prob.set_lambda_pts(0.7)
    p = torch.from_numpy(np.ascontiguousarray(fd.params, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(p)
    with pytest.raises(RuntimeError):
        prob.estimate_lambda_pts(p)
    prob.close()
    ref = copy.copy(fd)
    ref.W = Wm
    check_deconv(ref, loss, grad.cpu().numpy(), lam_pts=0.7)


def test_weight_map_in_a_batch_and_toggle_needs_recreate():
    from paper_2402_08725_gb300.binding import Batch, Problem
    fields = [syn.small_deconv(seed=2700 + i, E=2 + i, N=24, f=2, K=15, M=1, J=3) for i in range(3)]
    probs = [Problem.from_field(fd, conv_mode="direct") for fd in fields]
    maps = [_map(np.random.default_rng(9 + i), fd.W, fd.F) for i, fd in enumerate(fields)]
    probs[0].set_weight_map(maps[0])
    probs[2].set_weight_map(maps[2])
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(3, dtype=torch.float64, device="cuda")
    batch.loss_and_grad(P, losses=losses)
    for i, (fd, pr) in enumerate(zip(fields, probs)):
        l_i, _ = pr.loss_and_grad(torch.from_numpy(fd.params).cuda())
        assert losses[i].item() == l_i
    probs[1].set_weight_map(maps[1])
    with pytest.raises(RuntimeError):
        batch.loss_and_grad(P, losses=losses)
    batch.close()
    for pr in probs:
        pr.close()


def test_bad_weight_maps_are_rejected():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=2800, E=2, N=16, f=2, K=9, M=1, J=3)
    prob = Problem.from_field(fd)
    Wm = _map(np.random.default_rng(1), fd.W, fd.F)
    bad = Wm.copy()
    bad[1, 3, 4] = -1.0
    with pytest.raises(RuntimeError):
        prob.set_weight_map(bad)
    bad[1, 3, 4] = np.inf
    with pytest.raises(RuntimeError):
        prob.set_weight_map(bad)
    with pytest.raises(ValueError):
        prob.set_weight_map(Wm[:1])
    prob.close()
    assert oracle is not None and loss_errors and rel_l2 and LOSS_RTOL and GRAD_RTOL
