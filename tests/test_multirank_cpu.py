"""World-size-2 gloo tests of the multi-rank paths (CPU only).

Two ways the work shards:
  * epochs of one field split across ranks: every term of the chi^2 and its
    gradient is epoch-local except dL/dh and dL/dc_k, which are sums over
    epochs; one all-reduce of the partial losses and gradients (and the prior,
    added once) gives the full result;
  * independent fields (the uneven batch) split across ranks: no collective on
    the data path; only the timing (max over ranks) is reduced, as bench.py does.
Both are checked with the FP64 oracle on two gloo ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _epoch_shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2402_08725_gb300 import synthetic as syn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fd = syn.small_deconv(seed=77, E=4, N=12, f=2, K=7, M=2, J=3, lam=0.9)
    E, N, f, M = fd.E, fd.N, fd.f, fd.M
    F = f * N
    h, a, c, dl, gm = syn.unpack_deconv(fd.params, E, N, f, M)
    sl = slice(rank * E // world, (rank + 1) * E // world)
    Es = sl.stop - sl.start
    P = syn.pack_deconv(h, a[sl], c, dl[sl], gm[sl])
    # chi^2 part only on every rank (lambda = 0); the prior is added once after the reduction
    L, _, g, _ = oracle.deconv_loss_grad(Es, N, f, fd.K, M, fd.J, 0.0, fd.d[sl], fd.sigma[sl], fd.s[sl], fd.W, P)
    shared = torch.from_numpy(np.concatenate([[L], g[:F * F], g[F * F + Es * M:F * F + Es * M + 2 * M]]))
    dist.all_reduce(shared)
    if rank == 0:
        prior, gprior = oracle.starlet_prior(h, fd.J, fd.lam, fd.W)
        out.put((float(shared[0]) + prior, (shared[1:1 + F * F].numpy() + gprior.ravel()),
                 shared[1 + F * F:].numpy()))
    dist.destroy_process_group()


def test_epoch_sharded_allreduce_equals_full_gradient():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_epoch_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    L_sh, gh_sh, gc_sh = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2402_08725_gb300 import synthetic as syn
    fd = syn.small_deconv(seed=77, E=4, N=12, f=2, K=7, M=2, J=3, lam=0.9)
    F = fd.F
    L, _, g, _ = oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W,
                                         fd.params)
    assert abs(L_sh - L) <= 1e-12 * abs(L)
    np.testing.assert_allclose(gh_sh, g[:F * F], rtol=1e-10, atol=1e-10)
    oc = F * F + fd.E * fd.M
    np.testing.assert_allclose(gc_sh, g[oc:oc + 2 * fd.M], rtol=1e-10)


def _field_shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2402_08725_gb300 import synthetic as syn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fields = [syn.small_deconv(seed=200 + i, E=2, N=10 + 2 * i, f=2, K=5, M=1, J=3) for i in range(4)]
    mine = fields[rank::world]
    losses = [oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W,
                                      fd.params, grad=False)[0] for fd in mine]
    # the only collective: the max of the per-rank times, as in bench.py
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out.put((rank, losses, float(t.item())))
    dist.destroy_process_group()


def test_field_sharding_needs_no_data_collective():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_field_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(2)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2402_08725_gb300 import synthetic as syn
    fields = [syn.small_deconv(seed=200 + i, E=2, N=10 + 2 * i, f=2, K=5, M=1, J=3) for i in range(4)]
    ref = [oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s, fd.W,
                                   fd.params, grad=False)[0] for fd in fields]
    got = {}
    for rank, losses, tmax in res:
        assert tmax == 2.0
        for j, L in enumerate(losses):
            got[rank + 2 * j] = L
    assert [got[i] for i in range(4)] == ref
