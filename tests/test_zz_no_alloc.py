"""The allocation-free entry point, sr_loss_and_grad_noalloc, called through the
C ABI: two calls in a row must give what the allocating entry point
(sr_create_problem + set_* + sr_loss_and_grad) gives, within the parity
tolerances of the other GPU tests.  It serves callers that cannot allocate
device memory (a pool fixed at start-up, a loop that must not block on the
allocator); its scratch is one fixed device array inside the library.

This file is collected last so that a failure here cannot hide another test's.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import GRAD_RTOL, LOSS_RTOL, deconv_blocks, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def _desc(nat, fd):
    d = nat.ProblemDesc()
    d.kind, d.n_epochs, d.data_n, d.supersampling = nat.SR_DECONV, fd.E, fd.N, fd.f
    d.psf_k, d.n_sources, d.n_scales, d.lam, d.conv_mode = fd.K, fd.M, fd.J, fd.lam, nat.SR_CONV_AUTO
    return d


@pytest.mark.parametrize("case", ["small", "config1", "ragged_f3", "wide_psf_f8"])
def test_noalloc_matches_allocating_entry_point_twice(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native as nat
    from paper_2402_08725_gb300.binding import Problem
    lib = nat.load()
    if case == "small":
        fd = syn.small_deconv(seed=61, E=3, N=40, f=2, K=15, M=2, J=3, lam=1.2)
    elif case == "config1":
        fd = syn.config1()
    elif case == "ragged_f3":
        fd = syn.small_deconv(seed=62, E=2, N=70, f=3, K=21, M=1, J=4, lam=0.7)
    else:
        # f = 8 with a 255-pixel PSF on an 8x8 stamp: many phases per tile, each needing a
        # wide kernel in shared memory; both entry points must pick phase groups that fit
        fd = syn.small_deconv(seed=63, E=2, N=8, f=8, K=255, M=1, J=3, lam=0.5)
    ref = Problem.from_field(fd)
    P = torch.from_numpy(fd.params).cuda()
    L_ref, g_ref = ref.loss_and_grad(P)
    g_ref = g_ref.cpu().numpy()
    ref.close()

    d = torch.from_numpy(fd.d).cuda()
    sig = torch.from_numpy(fd.sigma).cuda()
    psf = torch.from_numpy(fd.s).cuda()
    W = np.ascontiguousarray(fd.W, dtype=np.float32)
    desc = _desc(nat, fd)
    stream = torch.cuda.current_stream()
    blocks = deconv_blocks(fd.E, fd.N, fd.f, fd.M)
    for _ in range(2):
        loss = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        grad = torch.full((fd.n_params,), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.sr_loss_and_grad_noalloc(ctypes.byref(desc), ctypes.c_void_p(d.data_ptr()),
                                          ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(psf.data_ptr()),
                                          ctypes.c_void_p(W.ctypes.data), ctypes.c_void_p(P.data_ptr()),
                                          ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
        nat.check(rc, "sr_loss_and_grad_noalloc")
        torch.cuda.synchronize()
        L = loss.item()
        g = grad.cpu().numpy()
        assert abs(L - L_ref) <= LOSS_RTOL * abs(L_ref)
        for name, sl in blocks.items():
            if sl.stop > sl.start:
                assert rel_l2(g[sl], g_ref[sl]) <= GRAD_RTOL, name


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native as nat
    lib = nat.load()
    d = nat.ProblemDesc()
    d.kind, d.n_epochs, d.data_n, d.supersampling = nat.SR_DECONV, 4000, 128, 2
    d.psf_k, d.n_sources, d.n_scales, d.lam, d.conv_mode = 64, 1, 4, 1.0, nat.SR_CONV_AUTO
    buf = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    W = np.ones(3, dtype=np.float32)
    rc = lib.sr_loss_and_grad_noalloc(ctypes.byref(d), p, p, p, ctypes.c_void_p(W.ctypes.data), p, p, p, None)
    assert rc == 2
    assert b"scratch" in lib.sr_last_error()


def test_noalloc_invalid_sigma_gives_nan_loss():
    """A sigma that is NaN or <= 0 has no inverse variance: the call, which returns no input
    check, reports it as a NaN loss (sigma = +inf still masks its pixel)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native as nat
    lib = nat.load()
    fd = syn.small_deconv(seed=64, E=2, N=24, f=2, K=11, M=1, J=3, lam=1.0)
    desc = _desc(nat, fd)
    P = torch.from_numpy(fd.params).cuda()
    d = torch.from_numpy(fd.d).cuda()
    psf = torch.from_numpy(fd.s).cuda()
    W = np.ascontiguousarray(fd.W, dtype=np.float32)
    stream = torch.cuda.current_stream()
    for bad, expect_nan in ((0.0, True), (-1.0, True), (float("nan"), True), (float("inf"), False)):
        sig_h = fd.sigma.copy()
        sig_h[1, 5, 7] = bad
        sig = torch.from_numpy(sig_h).cuda()
        loss = torch.zeros((), dtype=torch.float64, device="cuda")
        grad = torch.zeros((fd.n_params,), dtype=torch.float32, device="cuda")
        rc = lib.sr_loss_and_grad_noalloc(ctypes.byref(desc), ctypes.c_void_p(d.data_ptr()),
                                          ctypes.c_void_p(sig.data_ptr()), ctypes.c_void_p(psf.data_ptr()),
                                          ctypes.c_void_p(W.ctypes.data), ctypes.c_void_p(P.data_ptr()),
                                          ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
        nat.check(rc, "sr_loss_and_grad_noalloc")
        torch.cuda.synchronize()
        assert np.isnan(loss.item()) == expect_nan, (bad, loss.item())
