"""GPU parity of the PSF-reconstruction loss and gradient, the optimiser step,
graph replay, checkpoint/resume and error reporting, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import check_psf, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _psf(pb, params=None):
    from paper_2402_08725_gb300.binding import Problem
    prob = Problem.from_psf(pb)
    P = pb.params if params is None else params
    loss, grad = prob.loss_and_grad(torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda())
    g = grad.cpu().numpy()
    prob.close()
    return loss, g


@pytest.mark.parametrize("S,N,f,J", [(3, 16, 2, 3), (2, 21, 3, 3), (4, 12, 1, 2), (5, 40, 2, 4)])
def test_psf_small_cases(S, N, f, J):
    pb = syn.small_psf(seed=S * 10 + N, S=S, N=N, f=f, J=J, lam=1.0)
    loss, g = _psf(pb)
    check_psf(pb, loss, g)


def test_psf_star_near_edge():
    pb = syn.small_psf(seed=3, S=2, N=16, f=2, J=3)
    b, al, be, a, c = syn.unpack_psf(pb.params.copy(), pb.S, pb.N, pb.f)
    c[0] = (6.7, -7.1)
    P = syn.pack_psf(b, al, be, a, c)
    loss, g = _psf(pb, P)
    check_psf(pb, loss, g, params=P)


def test_config2_full_size():
    pb = syn.config2()
    loss, g = _psf(pb)
    r = check_psf(pb, loss, g)
    print("config2", r)


# --- optimiser --------------------------------------------------------------------------

def _lr(fd):
    return (1e-2, 0.05 * float(np.mean(fd.params[fd.F ** 2:fd.F ** 2 + fd.E * fd.M])) + 1.0, 1e-3, 1e-3, 1e-2)


def _oracle_steps(fd, n, lr_groups, kind=oracle.ADABELIEF, beta1=0.9, beta2=0.999, eps=1e-16):
    from tests._helpers import deconv_blocks
    blocks = deconv_blocks(fd.E, fd.N, fd.f, fd.M)
    P = fd.params.astype(np.float64).copy()
    lr = np.zeros(P.size)
    lo, hi = np.full(P.size, -np.inf), np.full(P.size, np.inf)
    for g, sl in enumerate(blocks.values()):
        lr[sl] = lr_groups[g]
    lo[blocks["a"]] = 0.0
    m, v = np.zeros(P.size), np.zeros(P.size)
    losses = []
    for t in range(1, n + 1):
        L, _, g, _ = oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s,
                                             fd.W, P)
        losses.append(L)
        oracle.optim_step(kind, P, g, m, v, t, lr, beta1, beta2, eps, lo, hi)
    return P, losses


@pytest.mark.parametrize("kind", ["adabelief", "adam"])
def test_optimiser_steps_match_oracle(kind):
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    fd = syn.small_deconv(seed=31, E=3, N=24, f=2, K=13, M=2, J=3, lam=1.0)
    lrs = _lr(fd)
    prob = Problem.from_field(fd)
    for n in (1, 10):
        prob.reset_optimizer()
        p = torch.from_numpy(fd.params).cuda()
        losses = torch.zeros(n, dtype=torch.float64, device="cuda")
        prob.step(p, n, optim_cfg(kind, lr=lrs), losses=losses)
        P_ref, L_ref = _oracle_steps(fd, n, lrs, kind=oracle.ADABELIEF if kind == "adabelief" else oracle.ADAM,
                                     eps=1e-16 if kind == "adabelief" else 1e-8)
        d = rel_l2(p.cpu().numpy() - fd.params, P_ref - fd.params.astype(np.float64))
        assert d <= 1e-3, (n, d)
        np.testing.assert_allclose(losses.cpu().numpy(), L_ref, rtol=1e-5)
    prob.close()


def test_graph_replay_equals_eager_and_checkpoint_resume():
    """sr_step runs captured graphs; stepping 6 + 6 with a saved/restored state
    gives bitwise the result of 12 uninterrupted steps."""
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    fd = syn.small_deconv(seed=33, E=4, N=32, f=2, K=15, M=2, J=3, lam=1.0)
    cfg = optim_cfg("adabelief", lr=_lr(fd))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        prob = Problem.from_field(fd, stream=s)
        pa = torch.from_numpy(fd.params).cuda()
        prob.step(pa, 12, cfg)
        prob.reset_optimizer()
        pb = torch.from_numpy(fd.params).cuda()
        prob.step(pb, 6, cfg)
        m, v, t = prob.get_state()
        m, v = m.clone(), v.clone()
        assert t == 6
        prob.reset_optimizer()
        prob.set_state(m, v, t)
        prob.step(pb, 6, cfg)
        s.synchronize()
        assert torch.equal(pa, pb)
        prob.close()
    # eager (legacy default stream, no graph) equals the graph replay
    prob2 = Problem.from_field(fd, stream=torch.cuda.default_stream())
    pc = torch.from_numpy(fd.params).cuda()
    prob2.step(pc, 12, cfg)
    torch.cuda.synchronize()
    assert torch.equal(pa, pc)
    prob2.close()


def test_steps_queued_without_read_back_on_two_streams():
    """step(sync=False) queues the steps without reading the loss back: a PSF fit and a batch
    stepped on two streams, forked from and joined to one stream by events, end bitwise where
    the synchronising calls end."""
    from paper_2402_08725_gb300.binding import Batch, Problem, optim_cfg
    fd = syn.small_deconv(seed=34, E=3, N=32, f=2, K=15, M=1, J=3, lam=1.0)
    pb = syn.small_psf(seed=35, S=3, N=16, f=2, J=3, lam=1.0)
    cfg = optim_cfg("adabelief", lr=_lr(fd))
    cfg_psf = optim_cfg("adabelief", lr=(1e-5, 1e-3, 10.0, 1e-3))
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    results = []
    for sync in (True, False):
        with torch.cuda.stream(main):
            prob = Problem.from_field(fd, stream=main)
            batch = Batch([prob], stream=main)
            psf = Problem.from_psf(pb, stream=side)
            P = torch.from_numpy(batch.pack([fd.params])).cuda()
            Q = torch.from_numpy(pb.params).cuda()
            torch.cuda.synchronize()
            fork, join = torch.cuda.Event(), torch.cuda.Event()
            for _ in range(4):
                fork.record(main)
                side.wait_event(fork)
                r_psf = psf.step(Q, 1, cfg_psf, sync=sync)
                join.record(side)
                r_b = batch.step(P, 1, cfg, sync=sync)
                main.wait_event(join)
                assert (r_psf is None and r_b is None) if not sync else np.isfinite(r_psf + r_b)
            main.synchronize()
            results.append((P.clone(), Q.clone()))
            batch.close()
            prob.close()
            psf.close()
    assert torch.equal(results[0][0], results[1][0]) and torch.equal(results[0][1], results[1][1])


def test_noiseless_recovery_on_gpu():
    """Data made by the oracle's model at known truth (no noise, lambda = 0):
    AdaBelief on (a, c) with h and delta held fixed recovers the truth."""
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    fd = syn.small_deconv(seed=21, E=3, N=14, f=2, K=9, M=2, J=3, lam=0.0)
    truth = fd.params.astype(np.float64)
    fd.d = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, truth).astype(np.float32)
    fd.sigma = np.full_like(fd.d, 3.0)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params, fd.E, fd.N, fd.f, fd.M)
    start = syn.pack_deconv(h, a * 1.2, c + 0.3, dl, gm)
    prob = Problem.from_field(fd)
    p = torch.from_numpy(start).cuda()
    prob.step(p, 1000, optim_cfg("adabelief", lr=(0.0, 0.02 * float(np.mean(a)), 0.01, 0.0, 0.0)))
    prob.step(p, 1000, optim_cfg("adabelief", lr=(0.0, 0.002 * float(np.mean(a)), 0.001, 0.0, 0.0)))
    _, a_r, c_r, _, _ = syn.unpack_deconv(p.cpu().numpy(), fd.E, fd.N, fd.f, fd.M)
    np.testing.assert_allclose(a_r, a, rtol=1e-3)
    np.testing.assert_allclose(c_r, c, atol=2e-3)
    prob.close()


def test_psf_optimiser_projection():
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    pb = syn.small_psf(seed=4, S=2, N=12, f=2, J=3)
    prob = Problem.from_psf(pb)
    p = torch.from_numpy(pb.params).cuda()
    prob.step(p, 3, optim_cfg("adam", lr=(1e-3, 100.0, 1e9, 1e-2)))
    b, al, be, a, c = syn.unpack_psf(p.cpu().numpy(), pb.S, pb.N, pb.f)
    assert al >= 1e-3 and be >= 1.001 - 1e-6
    assert np.all(a >= 0.0)
    prob.close()


def test_psf_optimiser_groups_move_separately():
    """Learning rate on one group of the layout at a time (b, Moffat alpha and beta, a, c): Adam's
    first step moves each variable by lr sign(g), so only the chosen group changes, by exactly
    its rate; and alpha keeps its own lower bound (1e-3), not beta's."""
    from paper_2402_08725_gb300.binding import Problem, optim_cfg
    pb = syn.small_psf(seed=6, S=2, N=12, f=2, J=3)
    F = pb.f * pb.N
    spans = [slice(0, F * F), slice(F * F, F * F + 2), slice(F * F + 2, F * F + 2 + pb.S),
             slice(F * F + 2 + pb.S, F * F + 2 + 3 * pb.S)]
    for gsel, sl in enumerate(spans):
        prob = Problem.from_psf(pb)
        p0 = pb.params.astype(np.float32)
        p = torch.from_numpy(p0.copy()).cuda()
        lr = [0.0] * 4
        lr[gsel] = 1e-3
        prob.step(p, 1, optim_cfg("adam", lr=tuple(lr)))
        moved = np.abs(p.cpu().numpy() - p0)
        others = np.ones(p0.size, dtype=bool)
        others[sl] = False
        assert np.all(moved[others] == 0.0), gsel
        mv, tol = moved[sl], 1e-6 + 2.0 * np.spacing(np.abs(p0[sl]))  # float32 rounding of x +- lr
        assert np.any(mv > 0) and np.all(np.abs(mv[mv > 0] - 1e-3) <= tol[mv > 0]), gsel
        prob.close()
    # alpha pushed below 1.001 stays there (its bound is 1e-3); beta is held at 1.001
    prob = Problem.from_psf(pb)
    q = pb.params.astype(np.float32).copy()
    q[F * F] = 1.0005
    q[F * F + 1] = 1.0015
    p = torch.from_numpy(q).cuda()
    prob.step(p, 1, optim_cfg("adam", lr=(0.0, 0.01, 0.0, 0.0)))
    out = p.cpu().numpy()
    assert out[F * F + 1] >= 1.001 - 1e-7 and abs(out[F * F] - 1.0005) == pytest.approx(0.01, rel=1e-3)
    prob.close()


# --- errors -------------------------------------------------------------------------------

def test_state_and_input_errors():
    from paper_2402_08725_gb300 import _native as nat
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=2, E=2, N=16, f=2, K=7, M=1, J=3)
    prob = Problem("deconv", fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam)
    p = torch.from_numpy(fd.params).cuda()
    with pytest.raises(nat.StarredError) as ei:
        prob.loss_and_grad(p)
    assert ei.value.status == "SR_ERR_STATE"
    with pytest.raises(nat.StarredError) as ei:
        prob.set_weights([1.0, float("inf")])
    assert ei.value.status == "SR_ERR_NONFINITE"
    prob.set_data(fd.d)
    prob.set_noise(fd.sigma)
    prob.set_psfs(fd.s)
    prob.set_weights(fd.W)
    loss, _ = prob.loss_and_grad(p)
    assert np.isfinite(loss)
    # inputs are checked on the device; the next call that returns a host value reports them
    bad = fd.d.copy()
    bad[1, 2, 3] = np.nan
    sig = fd.sigma.copy()
    sig[0, 0, 0] = -1.0
    psf = fd.s.copy()
    psf[0, 1, 1] = np.inf
    for setter, good, badv in ((prob.set_data, fd.d, bad), (prob.set_noise, fd.sigma, sig),
                               (prob.set_psfs, fd.s, psf)):
        for as_dev in (False, True):
            setter(torch.from_numpy(badv).cuda() if as_dev else badv)
            with pytest.raises(nat.StarredError) as ei:
                prob.loss_and_grad(p)
            assert ei.value.status == "SR_ERR_NONFINITE"
            setter(good)
            loss2, _ = prob.loss_and_grad(p)
            assert loss2 == loss
    psf_prob = Problem("psf", 2, 16, 2, J=3)
    with pytest.raises(nat.StarredError) as ei:
        psf_prob.set_psfs(np.ones(psf_prob.E * psf_prob.K * psf_prob.K, dtype=np.float32))
    assert ei.value.status == "SR_ERR_STATE"
    psf_prob.close()
    prob.close()


@pytest.mark.gpu
def test_measured_fp32_peak_is_physical():
    """The FMA microbenchmark (the direct form's roofline denominator) lands between a quarter of
    the nominal FP32 rate and just above it (SMs x 128 lanes x 2 FLOP x maximum SM clock)."""
    import torch
    from paper_2402_08725_gb300.binding import measure_fp32_peak
    props = torch.cuda.get_device_properties(0)
    clock_mhz = 2070.0
    try:
        import json, os
        with open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "MEASURED_PEAKS.json")) as fh:
            clock_mhz = float(json.load(fh).get("sm_max_mhz", clock_mhz))
    except OSError:
        pass
    nominal = props.multi_processor_count * 128 * 2 * clock_mhz * 1e6 / 1e12
    t = measure_fp32_peak()
    assert 0.25 * nominal < t < 1.05 * nominal, (t, nominal)


def test_psf_model_matches_oracle_moffat_plus_grid():
    """sr_psf_model: s = Moffat(alpha, beta) + b, against the oracle's Moffat (Eq. 2)."""
    from paper_2402_08725_gb300.binding import Problem
    pb = syn.small_psf(51, S=2, N=20, f=2, J=3)
    F = pb.f * pb.N
    p = Problem.from_psf(pb)
    P = pb.params.astype(np.float64)
    s = p.psf_model(torch.from_numpy(P.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    m, _, _ = oracle.moffat(F, float(np.float32(P[F * F])), float(np.float32(P[F * F + 1])))
    ref = m + P[:F * F].astype(np.float32).reshape(F, F)
    assert np.max(np.abs(s - ref)) <= 1e-6 * np.max(np.abs(ref))
    p.close()
