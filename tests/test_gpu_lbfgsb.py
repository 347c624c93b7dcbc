"""GPU parity of L-BFGS-B (sr_lbfgsb) against the FP64 oracle L-BFGS-B driven by the FP64 oracle
loss.  The device evaluates the loss and gradient in FP32 (gradient within 1e-4 relative L2 of
the oracle's), so the two runs take the same decisions while the iterates agree to about that
precision: the loss of every iterate within 1e-4 relative of the starting loss's scale, the final
parameters within 2e-3 relative L2 after a few iterations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import lbfgsb as olb  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _deconv_fun(fd, d=None):
    d = fd.d if d is None else d

    def fun(x):
        L, _, g, _ = oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, d, fd.sigma, fd.s, fd.W, x)
        return L, g
    return fun


def _bounds_deconv(fd):
    F = fd.F
    n = fd.params.size
    lo = np.full(n, -np.inf)
    lo[F * F:F * F + fd.E * fd.M] = 0.0
    return lo, np.full(n, np.inf)


def _compare(ref, gpu, x_gpu):
    assert gpu["iterations"] == ref["iterations"], (gpu, ref["status"])
    scale = abs(ref["history"][0])
    np.testing.assert_allclose(gpu["history"], ref["history"], rtol=0, atol=1e-4 * scale)
    assert np.linalg.norm(x_gpu - ref["x"]) <= 2e-3 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_lbfgsb_matches_oracle_on_a_deconvolution_field(mode):
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(41, E=3, N=12, f=2, K=9, M=2, J=3, lam=0.5)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    start = syn.pack_deconv(0.7 * h, 1.3 * a, c + 0.15, dl, gm).astype(np.float32).astype(np.float64)
    lo, hi = _bounds_deconv(fd)
    ref = olb.lbfgsb(_deconv_fun(fd), start, lo, hi, m=5, max_iter=6, pgtol=0.0, factr=0.0)
    p = Problem.from_field(fd, conv_mode=mode)
    P = torch.from_numpy(start.astype(np.float32)).cuda()
    gpu = p.lbfgsb(P, max_iter=6, m=5, pgtol=0.0, factr=0.0)
    _compare(ref, gpu, P.cpu().numpy().astype(np.float64))
    assert np.all(np.diff(gpu["history"]) < 0)  # every accepted step satisfies the Armijo condition
    p.close()


def test_lbfgsb_keeps_an_amplitude_at_its_bound():
    """Noiseless data in which source 1 is absent from epoch 0: from a negative start that
    amplitude is clipped to 0 and the bound stays active, on both sides."""
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(42, E=3, N=12, f=2, K=9, M=2, J=3, lam=0.0)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    a[0, 1] = 0.0
    truth = syn.pack_deconv(h, a, c, dl, gm).astype(np.float32).astype(np.float64)
    d = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, truth).astype(np.float32)
    a0 = a.copy()
    a0[0, 1] = -50.0
    a0[1:] *= 1.2
    start = syn.pack_deconv(h, a0, c, dl, gm).astype(np.float32).astype(np.float64)
    lo, hi = _bounds_deconv(fd)
    ref = olb.lbfgsb(_deconv_fun(fd, d.astype(np.float64)), start, lo, hi, m=5, max_iter=5, pgtol=0.0, factr=0.0)
    p = Problem("deconv", fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, 0.0)
    p.set_data(d)
    p.set_noise(fd.sigma)
    p.set_psfs(fd.s)
    p.set_weights(fd.W)
    P = torch.from_numpy(start.astype(np.float32)).cuda()
    gpu = p.lbfgsb(P, max_iter=5, m=5, pgtol=0.0, factr=0.0)
    x = P.cpu().numpy().astype(np.float64)
    _compare(ref, gpu, x)
    ia = fd.F ** 2 + 1  # a[0, 1]
    assert x[ia] == 0.0 and ref["x"][ia] == 0.0
    assert np.all(x[fd.F ** 2:fd.F ** 2 + fd.E * fd.M] >= 0.0)
    p.close()


def test_lbfgsb_matches_oracle_on_a_psf_fit():
    from paper_2402_08725_gb300.binding import Problem
    pb = syn.small_psf(43, S=3, N=12, f=2, J=3, lam=0.5)
    F = pb.f * pb.N
    start = pb.params.astype(np.float64).copy()
    start[:F * F] *= 0.5
    start[F * F] *= 1.2     # alpha
    start[F * F + 1] = 1.5  # beta
    start = start.astype(np.float32).astype(np.float64)
    n = start.size
    lo = np.full(n, -np.inf)
    lo[F * F] = 1e-3
    lo[F * F + 1] = 1.001
    lo[F * F + 2:F * F + 2 + pb.S] = 0.0

    def fun(x):
        L, _, g = oracle.psf_loss_grad(pb.S, pb.N, pb.f, pb.J, pb.lam, pb.t, pb.sigma, pb.W, x)
        return L, g
    ref = olb.lbfgsb(fun, start, lo, np.full(n, np.inf), m=4, max_iter=5, pgtol=0.0, factr=0.0)
    p = Problem.from_psf(pb)
    P = torch.from_numpy(start.astype(np.float32)).cuda()
    gpu = p.lbfgsb(P, max_iter=5, m=4, pgtol=0.0, factr=0.0)
    _compare(ref, gpu, P.cpu().numpy().astype(np.float64))
    p.close()


def test_lbfgsb_stops_on_its_criteria_and_rejects_bad_configurations():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(44, E=2, N=12, f=2, K=9, M=1, J=3, lam=0.5)
    p = Problem.from_field(fd)
    P = torch.from_numpy(fd.params.astype(np.float32)).cuda()
    r = p.lbfgsb(P, max_iter=0)
    assert r["iterations"] == 0 and r["status"] == "max_iter" and r["evaluations"] == 1
    r = p.lbfgsb(P, max_iter=200, pgtol=1e30)
    assert r["status"] == "pgtol" and r["iterations"] == 0
    r = p.lbfgsb(P, max_iter=200, factr=1e14)
    assert r["status"] in ("factr", "pgtol", "line_search") and r["iterations"] < 200
    with pytest.raises(RuntimeError, match="SR_ERR_ARG"):
        p.lbfgsb(P, m=11)
    with pytest.raises(RuntimeError, match="SR_ERR_ARG"):
        p.lbfgsb(P, pgtol=-1.0)
    p.close()


def test_batch_lbfgsb_matches_oracle_on_the_sum_of_fields():
    """sr_batch_lbfgsb: L-BFGS-B on the total loss of three fields of different shapes (one
    without point sources), each with its own amplitude bounds, against the oracle L-BFGS-B on
    the concatenated problem."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    fields = [syn.small_deconv(60, E=3, N=12, f=2, K=9, M=2, J=3, lam=0.5),
              syn.small_deconv(61, E=2, N=16, f=2, K=9, M=0, J=3, lam=0.5),
              syn.small_deconv(62, E=4, N=12, f=2, K=9, M=1, J=3, lam=0.5)]
    probs = [Problem.from_field(fd) for fd in fields]
    b = Batch(probs)
    starts = []
    for fd in fields:
        h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
        starts.append(syn.pack_deconv(0.7 * h, 1.3 * a, c + 0.15, dl, gm))
    x0 = b.pack(starts).astype(np.float64)
    lo = np.full(x0.size, -np.inf)
    for fd, o in zip(fields, b.offsets):
        lo[o + fd.F ** 2:o + fd.F ** 2 + fd.E * fd.M] = 0.0
    funs = [_deconv_fun(fd) for fd in fields]

    def total(x):
        L, g = 0.0, np.zeros_like(x)
        for fd, o, fn in zip(fields, b.offsets, funs):
            n = fd.params.size
            Li, gi = fn(x[o:o + n])
            L += Li
            g[o:o + n] = gi
        return L, g
    ref = olb.lbfgsb(total, x0, lo, np.full(x0.size, np.inf), m=5, max_iter=5, pgtol=0.0, factr=0.0)
    P = torch.from_numpy(x0.astype(np.float32)).cuda()
    gpu = b.lbfgsb(P, max_iter=5, m=5, pgtol=0.0, factr=0.0)
    _compare(ref, gpu, P.cpu().numpy().astype(np.float64))
    b.close()
    for p in probs:
        p.close()


def test_lbfgsb_with_a_memory_of_one_pair():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(45, E=2, N=12, f=2, K=9, M=1, J=3, lam=0.5)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
    start = syn.pack_deconv(0.8 * h, 1.2 * a, c - 0.1, dl, gm).astype(np.float32).astype(np.float64)
    lo, hi = _bounds_deconv(fd)
    ref = olb.lbfgsb(_deconv_fun(fd), start, lo, hi, m=1, max_iter=5, pgtol=0.0, factr=0.0)
    p = Problem.from_field(fd)
    P = torch.from_numpy(start.astype(np.float32)).cuda()
    gpu = p.lbfgsb(P, max_iter=5, m=1, pgtol=0.0, factr=0.0)
    _compare(ref, gpu, P.cpu().numpy().astype(np.float64))
    p.close()


def _field_starts():
    """Three fields of different shapes (one without point sources, one whose source 1 is absent
    from epoch 0 in noiseless data and starts negative, so its bound becomes active)."""
    fields = [syn.small_deconv(70, E=3, N=12, f=2, K=9, M=2, J=3, lam=0.5),
              syn.small_deconv(71, E=2, N=16, f=2, K=9, M=0, J=3, lam=0.8),
              syn.small_deconv(72, E=3, N=12, f=2, K=9, M=2, J=3, lam=0.0)]
    starts = []
    for i, fd in enumerate(fields):
        h, a, c, dl, gm = syn.unpack_deconv(fd.params.astype(np.float64), fd.E, fd.N, fd.f, fd.M)
        if i == 2:
            a[0, 1] = 0.0
            truth = syn.pack_deconv(h, a, c, dl, gm).astype(np.float32).astype(np.float64)
            fd.d = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, truth).astype(np.float32)
            a0 = a.copy()
            a0[0, 1] = -50.0
            a0[1:] *= 1.2
            starts.append(syn.pack_deconv(h, a0, c, dl, gm))
        else:
            starts.append(syn.pack_deconv(0.7 * h, 1.3 * a, c + 0.15, dl, gm))
    return fields, [s.astype(np.float32).astype(np.float64) for s in starts]


def _run_fields(fields, starts, mode="auto", **kw):
    from paper_2402_08725_gb300.binding import Batch, Problem
    probs = [Problem.from_field(fd, conv_mode=mode) for fd in fields]
    b = Batch(probs)
    P = torch.from_numpy(b.pack(starts).astype(np.float32)).cuda()
    res, rounds = b.lbfgsb_fields(P, **kw)
    x = P.cpu().numpy().astype(np.float64)
    xs = [x[o:o + fd.params.size] for fd, o in zip(fields, b.offsets)]
    b.close()
    for p in probs:
        p.close()
    return res, rounds, xs


@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_batch_lbfgsb_fields_match_the_oracle_field_by_field(mode):
    """sr_batch_lbfgsb_fields: one L-BFGS-B per field, advanced together, against the oracle
    L-BFGS-B run on each field's own loss."""
    fields, starts = _field_starts()
    res, rounds, xs = _run_fields(fields, starts, mode, max_iter=6, m=5, pgtol=0.0, factr=0.0)
    for fd, s, r, x in zip(fields, starts, res, xs):
        lo, hi = _bounds_deconv(fd)
        ref = olb.lbfgsb(_deconv_fun(fd), s, lo, hi, m=5, max_iter=6, pgtol=0.0, factr=0.0)
        _compare(ref, r, x)
        assert np.all(np.diff(r["history"]) < 0)
    F, EM = fields[2].F, fields[2].E * fields[2].M
    amps = xs[2][F * F:F * F + EM]
    assert np.all(amps >= 0.0)
    assert amps[1] <= 1e-9 * np.abs(amps).max()  # the amplitude absent from the data stays at its bound
    assert rounds >= 6


def test_batch_lbfgsb_fields_do_not_depend_on_their_batch_mates():
    """Each field's run in a batch equals its run in a batch of its own, bit for bit, also when
    the fields stop at different iterations on their own criteria."""
    fields, starts = _field_starts()
    kw = dict(max_iter=40, m=4, pgtol=0.0, factr=1e13)
    res, rounds, xs = _run_fields(fields, starts, "direct", **kw)
    iters = set()
    for i in range(len(fields)):
        r1, _, x1 = _run_fields([fields[i]], [starts[i]], "direct", **kw)
        assert r1[0]["iterations"] == res[i]["iterations"]
        assert r1[0]["status"] == res[i]["status"]
        assert np.array_equal(r1[0]["history"], res[i]["history"])
        assert np.array_equal(x1[0], xs[i])
        iters.add(res[i]["iterations"])
    assert len(iters) > 1, res  # the fields stopped at different iterations


def test_batch_lbfgsb_fields_stopping_criteria():
    fields, starts = _field_starts()
    res, _, _ = _run_fields(fields, starts, max_iter=0)
    assert all(r["iterations"] == 0 and r["status"] == "max_iter" for r in res)
    res, _, _ = _run_fields(fields, starts, max_iter=50, pgtol=1e30)
    assert all(r["iterations"] == 0 and r["status"] == "pgtol" for r in res)
    from paper_2402_08725_gb300.binding import Batch, Problem
    p = Problem.from_field(fields[0])
    b = Batch([p])
    P = torch.from_numpy(b.pack([starts[0]]).astype(np.float32)).cuda()
    with pytest.raises(RuntimeError):
        b.lbfgsb_fields(P, m=11)
    b.close()
    p.close()
