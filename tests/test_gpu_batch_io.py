"""Batched input set-up (sr_batch_set_data / _noise / _psfs): the same effect as the members'
own set-up calls, bit for bit, for members of both convolution forms and of different shapes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _fields():
    return [syn.small_deconv(70, E=3, N=16, f=2, K=13, M=2, J=3, lam=0.5),
            syn.small_deconv(71, E=5, N=24, f=2, K=11, M=1, J=4, lam=0.5),
            syn.small_deconv(72, E=2, N=12, f=3, K=9, M=0, J=3, lam=0.5),
            syn.small_deconv(73, E=4, N=32, f=2, K=15, M=1, J=4, lam=0.5)]


def _batch(fields, modes):
    from paper_2402_08725_gb300.binding import Batch, Problem
    probs = [Problem.from_field(fd, conv_mode=m) for fd, m in zip(fields, modes)]
    return probs, Batch(probs)


def _eval(b, fields):
    P = torch.from_numpy(b.pack([fd.params for fd in fields])).cuda()
    lt = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    tot, g = b.loss_and_grad_host(P.cpu().numpy())
    return tot, g


@pytest.mark.parametrize("on_device", [False, True])
def test_batch_set_equals_member_set(on_device):
    fields = _fields()
    modes = ["fft", "direct", "fft", "auto"]
    rng = np.random.default_rng(5)
    # new inputs: scaled data, perturbed noise, other PSFs (each member's PSFs of another seed)
    new_d = [(fd.d * 1.1 + 0.5).astype(np.float32) for fd in fields]
    new_s = [(fd.sigma * rng.uniform(0.9, 1.1, fd.sigma.shape)).astype(np.float32) for fd in fields]
    new_p = [syn.moffat_stack(fd.K, rng.uniform(2, 3, fd.E), rng.uniform(2, 4, fd.E)) for fd in fields]
    new_s[0][0, 1, 1] = np.inf  # a masked pixel
    pa, ba = _batch(fields, modes)
    for pr, d, s, p in zip(pa, new_d, new_s, new_p):
        pr.set_data(d)
        pr.set_noise(s)
        pr.set_psfs(p)
    ta, ga = _eval(ba, fields)
    pb, bb = _batch(fields, modes)
    cat = lambda xs: np.concatenate([x.ravel() for x in xs]).astype(np.float32)
    conv = (lambda a: torch.from_numpy(a).cuda()) if on_device else (lambda a: a)
    bb.set_data(conv(cat(new_d)))
    bb.set_noise(conv(cat(new_s)))
    bb.set_psfs(conv(cat(new_p)))
    tb, gb = _eval(bb, fields)
    assert ta == tb and np.array_equal(ga, gb)
    assert bb.field_forms() == ba.field_forms()
    for x in (ba, bb):
        x.close()
    for pr in pa + pb:
        pr.close()


def test_batch_set_reports_bad_inputs():
    fields = _fields()
    pr, b = _batch(fields, ["auto"] * len(fields))
    d = np.concatenate([fd.d.ravel() for fd in fields]).astype(np.float32)
    d[d.size // 2] = np.nan
    b.set_data(d)
    with pytest.raises(RuntimeError, match="SR_ERR_NONFINITE"):
        _eval(b, fields)
    b.set_data(np.concatenate([fd.d.ravel() for fd in fields]).astype(np.float32))
    s = np.concatenate([fd.sigma.ravel() for fd in fields]).astype(np.float32)
    s[3] = -1.0
    b.set_noise(s)
    with pytest.raises(RuntimeError, match="SR_ERR_NONFINITE"):
        _eval(b, fields)
    b.set_noise(np.concatenate([fd.sigma.ravel() for fd in fields]).astype(np.float32))
    tot, _ = _eval(b, fields)
    assert np.isfinite(tot)
    b.close()
    for p in pr:
        p.close()


def test_pipelined_host_steps_equal_synchronous_ones():
    """Steps queued with sr_batch_loss_and_grad_host_async, each with its own inputs (three sets
    of data, noise, PSFs and parameters in turn, from page-locked memory), give the synchronous
    call's loss and gradient for those inputs bit for bit: the next step's staged copies overlap
    this step's evaluation without overwriting what it reads."""
    fields = _fields()
    modes = ["fft", "direct", "fft", "auto"]
    rng = np.random.default_rng(9)
    cat = lambda xs: np.concatenate([x.ravel() for x in xs]).astype(np.float32)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    sets = []
    for k in range(3):
        d = cat([fd.d * (1.0 + 0.1 * k) + k for fd in fields])
        s = cat([fd.sigma * rng.uniform(0.9, 1.1, fd.sigma.shape) for fd in fields])
        p = cat([syn.moffat_stack(fd.K, rng.uniform(2, 3, fd.E), rng.uniform(2, 4, fd.E)) for fd in fields])
        q = cat([fd.params * (1.0 + 0.05 * k) for fd in fields])
        sets.append((pin(d), pin(s), pin(p), pin(q)))
    pr, b = _batch(fields, modes)
    ref = []
    for d, s, p, q in sets:
        b.set_psfs(p)
        b.set_data(d)
        b.set_noise(s)
        tot, g = b.loss_and_grad_host(q.numpy())
        ref.append((tot, g.copy()))
    order = [0, 1, 2, 1, 0, 2]
    outs = [(torch.empty(b.n_params, dtype=torch.float32).pin_memory().numpy(),
             torch.empty(1, dtype=torch.float64).pin_memory().numpy()) for _ in order]
    for k, (g, t) in zip(order, outs):
        d, s, p, q = sets[k]
        b.set_psfs(p)
        b.set_data(d)
        b.set_noise(s)
        b.loss_and_grad_host_async(q.numpy(), g, t)
    b.sync()
    for k, (g, t) in zip(order, outs):
        assert t[0] == ref[k][0] and np.array_equal(g, ref[k][1]), k
    b.close()
    for p_ in pr:
        p_.close()


def test_pipelined_sync_reports_bad_inputs():
    fields = _fields()
    pr, b = _batch(fields, ["auto"] * len(fields))
    d = np.concatenate([fd.d.ravel() for fd in fields]).astype(np.float32)
    d[3] = np.inf
    q = b.pack([fd.params for fd in fields])
    g = np.empty(b.n_params, dtype=np.float32)
    t = np.empty(1, dtype=np.float64)
    b.set_data(d)
    b.loss_and_grad_host_async(q, g, t)
    with pytest.raises(RuntimeError, match="SR_ERR_NONFINITE"):
        b.sync()
    b.close()
    for p_ in pr:
        p_.close()


def test_batch_set_scalar_paths_and_unaligned_host_buffers():
    """Packed offsets that are not multiples of 4 (odd stamp and PSF sizes) take the per-element
    set-up path, and page-locked parameter / gradient buffers that start off a 16-byte boundary
    the per-element host-copy kernel; both give the members' own set-up and the device-buffer
    evaluation bit for bit."""
    fields = [syn.small_deconv(80, E=3, N=15, f=2, K=13, M=1, J=3, lam=0.5),
              syn.small_deconv(81, E=2, N=17, f=2, K=9, M=0, J=3, lam=0.5)]
    modes = ["fft", "direct"]
    rng = np.random.default_rng(12)
    new_d = [(fd.d * 0.9 + 1.0).astype(np.float32) for fd in fields]
    new_s = [(fd.sigma * rng.uniform(0.9, 1.1, fd.sigma.shape)).astype(np.float32) for fd in fields]
    new_p = [syn.moffat_stack(fd.K, rng.uniform(2, 3, fd.E), rng.uniform(2, 4, fd.E)) for fd in fields]
    pa, ba = _batch(fields, modes)
    for pr, d, s, p in zip(pa, new_d, new_s, new_p):
        pr.set_data(d)
        pr.set_noise(s)
        pr.set_psfs(p)
    ta, ga = _eval(ba, fields)
    pb, bb = _batch(fields, modes)
    cat = lambda xs: np.concatenate([x.ravel() for x in xs]).astype(np.float32)
    bb.set_data(cat(new_d))
    bb.set_noise(cat(new_s))
    bb.set_psfs(cat(new_p))
    tb, gb = _eval(bb, fields)
    assert ta == tb and np.array_equal(ga, gb)
    # the same evaluation from page-locked buffers one float past a 16-byte boundary
    n = bb.n_params
    qbuf = torch.empty(n + 1, dtype=torch.float32).pin_memory()
    qbuf[1:] = torch.from_numpy(bb.pack([fd.params for fd in fields]))
    gbuf = torch.empty(n + 1, dtype=torch.float32).pin_memory()
    tbuf = torch.empty(1, dtype=torch.float64).pin_memory()
    q, g, t = qbuf.numpy()[1:], gbuf.numpy()[1:], tbuf.numpy()
    assert q.ctypes.data % 16 != 0 and g.ctypes.data % 16 != 0
    bb.loss_and_grad_host_async(q, g, t)
    bb.sync()
    assert t[0] == tb and np.array_equal(g, gb)
    tc, gc = bb.loss_and_grad_host(q, g)
    assert tc == tb and np.array_equal(gc, gb)
    for x in (ba, bb):
        x.close()
    for pr in pa + pb:
        pr.close()


@pytest.mark.parametrize("kind", ["deconv", "psf"])
def test_problem_async_host_evaluation_equals_synchronous(kind):
    """sr_loss_and_grad_host_async + sr_sync give sr_loss_and_grad_host's loss and gradient bit
    for bit, with the inputs set from page-locked memory (copied by kernels) in between."""
    from paper_2402_08725_gb300.binding import Problem
    if kind == "deconv":
        fd = syn.small_deconv(90, E=4, N=16, f=2, K=13, M=2, J=3, lam=0.5)
        pr = Problem.from_field(fd)
        d, s, q0 = fd.d, fd.sigma, fd.params
    else:
        fd = syn.small_psf(seed=91, S=3, N=16, f=2, J=3, lam=1.0)
        pr = Problem.from_psf(fd)
        d, s, q0 = fd.t, fd.sigma, fd.params
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    sets = [(pin(d * (1.0 + 0.2 * k)), pin(s), pin(q0 * (1.0 + 0.01 * k)).numpy()) for k in range(3)]
    ref = []
    for dk, sk, qk in sets:
        pr.set_data(dk)
        pr.set_noise(sk)
        loss, g = pr.loss_and_grad_host(qk)
        ref.append((loss, g.copy()))
    outs = [(torch.empty(pr.n_params, dtype=torch.float32).pin_memory().numpy(),
             torch.empty(1, dtype=torch.float64).pin_memory().numpy()) for _ in sets]
    for (dk, sk, qk), (g, l) in zip(sets, outs):
        pr.set_data(dk)
        pr.set_noise(sk)
        pr.loss_and_grad_host_async(qk, g, l)
    pr.sync()
    for (g, l), (rl, rg) in zip(outs, ref):
        assert l[0] == rl and np.array_equal(g, rg)
    pr.close()


def test_queued_evaluation_from_pageable_buffers():
    """sr_batch_loss_and_grad_host_async with ordinary (pageable) numpy buffers takes the copy
    path instead of the mapped-memory kernels and still gives the synchronous result bit for bit;
    sr_batch_sync with nothing queued returns at once."""
    fields = _fields()
    pr, b = _batch(fields, ["fft", "direct", "fft", "auto"])
    b.sync()
    q = b.pack([fd.params for fd in fields])
    tot, gref = b.loss_and_grad_host(q)
    g = np.empty(b.n_params, dtype=np.float32)
    t = np.empty(1, dtype=np.float64)
    b.loss_and_grad_host_async(q, g, t)
    b.sync()
    assert t[0] == tot and np.array_equal(g, gref)
    with pytest.raises(TypeError):
        b.loss_and_grad_host_async(q.astype(np.float64), g, t)
    b.close()
    for p_ in pr:
        p_.close()
