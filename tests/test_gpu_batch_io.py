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
