"""GPU parity of the joint-deconvolution loss and gradient (fused D-folded path and
the plain per-epoch path) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402
from tests._helpers import check_deconv, deconv_blocks  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_08725_gb300 import _native
    _native.load()
    yield


def _run(fd, params=None, conv_mode="auto"):
    from paper_2402_08725_gb300.binding import Problem
    prob = Problem.from_field(fd, conv_mode=conv_mode)
    P = fd.params if params is None else params
    p = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    loss, grad = prob.loss_and_grad(p)
    g = grad.cpu().numpy()
    prob.close()
    return loss, g


# (E, N, f, K, M, J): tiles of 64 plus ragged tails, odd/even K, f = 1, 2, 3, M = 0
SMALL = [
    (3, 24, 2, 15, 2, 3),
    (2, 80, 2, 21, 3, 4),
    (2, 20, 3, 17, 1, 3),
    (2, 16, 1, 9, 2, 3),
    (2, 30, 2, 64, 2, 4),
    (3, 37, 2, 12, 0, 3),
    (1, 8, 2, 5, 1, 2),
    (2, 70, 3, 30, 2, 5),
]


@pytest.mark.parametrize("E,N,f,K,M,J", SMALL)
@pytest.mark.parametrize("mode", ["direct", "plain", "fft"])
def test_small_cases_match_oracle(E, N, f, K, M, J, mode):
    fd = syn.small_deconv(seed=100 + N + K, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.5)
    loss, g = _run(fd, conv_mode=mode)
    check_deconv(fd, loss, g)


# The transform sizes that carry most of the config-4 epoch-pixels: L = 80 / 120 / 144 for
# N = 64 / 96 / 128 with K = 64, f = 2.  M = 1 takes the one-source paths (and epochs side by
# side where their buffers fit), M = 4 the up-to-four-source path.  E = 19: one full 16-epoch
# work item and a 3-epoch item whose last group is partial.
HEADLINE = [(64, 1), (64, 4), (96, 1), (96, 4), (128, 1), (128, 4)]


@pytest.mark.parametrize("N,M", HEADLINE)
def test_headline_transform_sizes_match_oracle(N, M):
    fd = syn.small_deconv(seed=700 + N + M, E=19, N=N, f=2, K=64, M=M, J=4, lam=1.5)
    loss, g = _run(fd, conv_mode="fft")
    r = check_deconv(fd, loss, g)
    print("headline fft", N, M, r)


# Transform sizes beyond shared memory (global-memory transforms, the config-5 form): L = 192 for
# N = 160, K = 63, f = 2, and for N = 140, K = 127, f = 3 (nine phases, odd pairing) with masked
# pixels, backgrounds and more sources than the in-shared-memory form takes.
@pytest.mark.parametrize("E,N,f,K,M,J", [(3, 160, 2, 63, 3, 4), (2, 140, 3, 127, 12, 4)])
def test_global_memory_transforms_match_oracle(E, N, f, K, M, J):
    fd = syn.small_deconv(seed=900 + N + K, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.2, pos_half=N / 5)
    fd.sigma[0, 10:20, 30:41] = np.inf
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    gm = np.linspace(-0.3, 0.4, fd.E)
    c[0] = (N / 2 - 1.3, -N / 2 + 1.7)   # window clipped by the grid
    P = syn.pack_deconv(h, a, c, dl, gm)
    loss, g = _run(fd, P, conv_mode="fft")
    r = check_deconv(fd, loss, g, params=P)
    print("global-memory transforms", (E, N, f, K, M), r)


def test_global_memory_transforms_batch_equals_single():
    """A batch with a global-memory field between in-shared-memory ones gives each field exactly
    its own evaluation."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    fields = [syn.small_deconv(seed=950, E=3, N=48, f=2, K=17, M=1, J=3),
              syn.small_deconv(seed=951, E=3, N=160, f=2, K=63, M=2, J=4),
              syn.small_deconv(seed=952, E=5, N=32, f=2, K=64, M=1, J=4)]
    probs = [Problem.from_field(fd, conv_mode="fft") for fd in fields]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    total, grad = batch.loss_and_grad(P, losses=losses)
    for i, (fd, pr) in enumerate(zip(fields, probs)):
        l_i, g_i = pr.loss_and_grad(torch.from_numpy(fd.params).cuda())
        o = batch.offsets[i]
        assert losses[i].item() == l_i
        assert torch.equal(grad[o:o + fd.n_params], g_i)
    batch.close()
    for pr in probs:
        pr.close()


def test_near_truth_config3_field_against_loss_itself():
    """A config-3 field (64x64, K = 64, 4 sources) whose data are the oracle's model at the
    evaluation point plus Gaussian noise of the field's sigma: the loss sits near its expected
    value 0.5 * npix, far below 0.5 * sum w d^2, and is checked against L itself."""
    fd = syn.config3(E=40)
    rng = np.random.default_rng(31)
    P = fd.params.astype(np.float32).astype(np.float64)
    model = oracle.deconv_model(fd.E, fd.N, fd.f, fd.K, fd.M, fd.s, P)
    fd.d = (model + fd.sigma * rng.standard_normal(model.shape)).astype(np.float32)
    for mode in ("direct", "fft"):
        loss, g = _run(fd, conv_mode=mode)
        r = check_deconv(fd, loss, g)
        npix = fd.E * fd.N * fd.N
        assert abs(2.0 * r["loss_ref"] / npix - 1.0) < 0.5, r
        print("near-truth config3", mode, r)


def test_masked_pixels_background_and_edge_source():
    fd = syn.small_deconv(seed=5, E=3, N=28, f=2, K=13, M=2, J=3, lam=0.8)
    fd.sigma[0, 3:9, 4:11] = np.inf
    fd.sigma[2, :, 0] = np.inf
    h, a, c, dl, gm = syn.unpack_deconv(fd.params.copy(), fd.E, fd.N, fd.f, fd.M)
    c[1] = (13.2, -13.4)   # near the corner: window clipped by the grid
    gm = np.array([0.3, -0.2, 0.1])
    P = syn.pack_deconv(h, a, c, dl, gm)
    for mode in ("direct", "plain", "fft"):
        loss, g = _run(fd, P, conv_mode=mode)
        check_deconv(fd, loss, g, params=P)


def test_lambda_zero_and_large():
    for lam in (0.0, 20.0):
        fd = syn.small_deconv(seed=9, E=2, N=32, f=2, K=17, M=1, J=4, lam=lam)
        for mode in ("direct", "fft"):
            loss, g = _run(fd, conv_mode=mode)
            check_deconv(fd, loss, g)


def test_config1_full_size():
    fd = syn.config1()
    for mode in ("direct", "plain", "fft"):
        loss, g = _run(fd, conv_mode=mode)
        r = check_deconv(fd, loss, g)
        print("config1", mode, r)


@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_config3_full_size(mode):
    """300 epochs of 64x64, f=2, K=64, 4 sources: all epochs in one persistent launch."""
    fd = syn.config3()
    loss, g = _run(fd, conv_mode=mode)
    r = check_deconv(fd, loss, g)
    print("config3", mode, r)


@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_repeatable_bitwise(mode):
    fd = syn.small_deconv(seed=4, E=5, N=48, f=2, K=21, M=2, J=4, lam=1.0)
    from paper_2402_08725_gb300.binding import Problem
    prob = Problem.from_field(fd, conv_mode=mode)
    p = torch.from_numpy(fd.params).cuda()
    l1, g1 = prob.loss_and_grad(p)
    g1 = g1.clone()
    l2, g2 = prob.loss_and_grad(p)
    assert l1 == l2
    assert torch.equal(g1, g2)
    prob.close()


def test_many_overlapping_sources_direct_form_deterministic():
    """40 point sources packed into a few pixels (their 16 x 16 windows overlap) in the direct
    form: every staged pixel adds its sources in index order, so repeated evaluations and a batch
    of copies give bitwise the single evaluation; the values match the oracle."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    fd = syn.small_deconv(seed=404, E=3, N=40, f=2, K=15, M=40, J=3, lam=1.0, pos_half=2.5)
    prob = Problem.from_field(fd, conv_mode="direct")
    p = torch.from_numpy(fd.params).cuda()
    l1, g1 = prob.loss_and_grad(p)
    g1 = g1.clone()
    l2, g2 = prob.loss_and_grad(p)
    assert l1 == l2 and torch.equal(g1, g2)
    check_deconv(fd, l1, g1.cpu().numpy())
    probs = [Problem.from_field(fd, conv_mode="direct") for _ in range(3)]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params] * 3)).cuda()
    losses = torch.empty(3, dtype=torch.float64, device="cuda")
    batch.loss_and_grad(P, losses=losses)
    grad = batch.loss_and_grad(P, losses=losses)[1]
    for i in range(3):
        assert losses[i].item() == l1
        o = batch.offsets[i]
        assert torch.equal(grad[o:o + fd.n_params], g1)
    batch.close()
    for q in probs + [prob]:
        q.close()


def test_batch_equals_single_fields_bitwise():
    """An uneven batch (sizes, epoch counts, starlet depths, and both the direct and the
    transform form) gives each field exactly the loss and gradient of its own
    single-problem evaluation."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    shapes = [(3, 32, 4), (5, 48, 5), (2, 64, 4), (4, 96, 6), (1, 20, 3)]
    fields = [syn.small_deconv(seed=50 + i, E=E, N=N, f=2, K=17, M=1, J=J, lam=1.0)
              for i, (E, N, J) in enumerate(shapes)]
    probs = [Problem.from_field(fd, conv_mode=("fft" if i % 2 else "direct")) for i, fd in enumerate(fields)]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    total, grad = batch.loss_and_grad(P, losses=losses)
    for i, (fd, pr) in enumerate(zip(fields, probs)):
        l_i, g_i = pr.loss_and_grad(torch.from_numpy(fd.params).cuda())
        o = batch.offsets[i]
        assert losses[i].item() == l_i
        assert torch.equal(grad[o:o + fd.n_params], g_i)
    assert abs(total - losses.sum().item()) <= 1e-12 * abs(total)
    batch.close()
    for pr in probs:
        pr.close()


def test_config4_full_batch_sampled_fields():
    """The full uneven batch of 256 fields in one evaluation; fields the oracle
    evaluates in seconds are checked against it (loss and gradient segments)."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    shapes = syn.config4_shapes()
    fields = syn.config4()
    probs = [Problem.from_field(fd) for fd in fields]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    total, grad = batch.loss_and_grad(P, losses=losses)
    assert np.isfinite(total)
    cost = [E * N * N for (N, E, J) in shapes]
    order = np.argsort(cost)
    picks = list(order[:3]) + [order[len(order) // 4]]
    # the two largest stamp sizes (transform sizes 120 and 144): the cheapest field of each,
    # and the N = 128 field of median epoch count
    for n in (96, 128):
        ids = sorted((shapes[i][1], i) for i in range(len(shapes)) if shapes[i][0] == n)
        picks.append(ids[0][1])
        if n == 128:
            picks.append(ids[len(ids) // 2][1])
    g_all = grad.cpu().numpy()
    ls = losses.cpu().numpy()
    for i in picks:
        fd = fields[i]
        o = batch.offsets[i]
        r = check_deconv(fd, float(ls[i]), g_all[o:o + fd.n_params])
        print("config4 field", i, shapes[i], r)
    batch.close()
    for pr in probs:
        pr.close()


def test_autograd_function():
    from paper_2402_08725_gb300.binding import Problem
    from paper_2402_08725_gb300.torch_ops import starred_loss
    fd = syn.small_deconv(seed=8, E=2, N=24, f=2, K=11, M=1, J=3, lam=1.0)
    prob = Problem.from_field(fd)
    p = torch.from_numpy(fd.params).cuda().requires_grad_(True)
    L = starred_loss(p, prob)
    (2.0 * L).backward()
    loss, g = prob.loss_and_grad(p.detach())
    assert abs(L.item() - loss) == 0.0
    assert torch.allclose(p.grad, 2.0 * g, rtol=0, atol=0)
    prob.close()


def test_host_buffer_entry_point_matches_device():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=12, E=3, N=32, f=2, K=13, M=2, J=3, lam=1.0)
    prob = Problem.from_field(fd)
    l_h, g_h = prob.loss_and_grad_host(fd.params)
    l_d, g_d = prob.loss_and_grad(torch.from_numpy(fd.params).cuda())
    assert l_h == l_d
    np.testing.assert_array_equal(g_h, g_d.cpu().numpy())
    prob.close()


def test_gradient_blocks_layout_matches_library():
    from paper_2402_08725_gb300.binding import Problem
    fd = syn.small_deconv(seed=1, E=3, N=16, f=2, K=7, M=2, J=3)
    prob = Problem.from_field(fd)
    lay = prob.layout()
    blocks = deconv_blocks(fd.E, fd.N, fd.f, fd.M)
    assert [(s.start, s.stop - s.start) for s in blocks.values()] == lay
    prob.close()


def test_config5_one_full_frame_matches_oracle():
    """JWST-like frame at full size: 512x512 data, f = 3 (1536x1536 model grid), 255x255 PSF,
    40 clumps, 6 starlet scales, one frame (the oracle evaluates it in about a minute)."""
    fd = syn.config5(E=1)
    loss, g = _run(fd)
    r = check_deconv(fd, loss, g)
    print("config5 frame", r)


def test_config5_six_frames_add_up():
    """All 6 frames in one evaluation (the benchmarked launch configuration): with the prior
    off, the loss and the shared-parameter gradients are the sums over single-frame
    evaluations — a property that holds at any size."""
    fd = syn.config5()
    fd.lam = 0.0
    loss6, g6 = _run(fd)
    h, a, c, dl, gm = syn.unpack_deconv(fd.params, fd.E, fd.N, fd.f, fd.M)
    F = fd.F
    tot, gh, gc = 0.0, np.zeros(F * F), np.zeros(2 * fd.M)
    for i in range(fd.E):
        one = syn.DeconvField(1, fd.N, fd.f, fd.K, fd.M, fd.J, 0.0, fd.d[i:i + 1], fd.sigma[i:i + 1],
                              fd.s[i:i + 1], fd.W, syn.pack_deconv(h, a[i:i + 1], c, dl[i:i + 1], gm[i:i + 1]))
        l1, g1 = _run(one)
        tot += l1
        gh += g1[:F * F]
        gc += g1[F * F + fd.M:F * F + 3 * fd.M]
    # the transform form carries two frames in one complex transform, so a frame's rounding
    # depends on the frame it is paired with: equal to FP32 rounding, far inside the parity bounds
    assert abs(loss6 - tot) <= 1e-7 * abs(tot)
    from tests._helpers import rel_l2
    assert rel_l2(g6[:F * F], gh) <= 1e-5
    oc = F * F + fd.E * fd.M
    assert rel_l2(g6[oc:oc + 2 * fd.M], gc) <= 1e-5


def test_autotuner_resolves_auto_fields_and_caches(tmp_path, monkeypatch):
    """AUTO fields whose shape fits both forms are timed once per shape; the choice is
    reported per field and written to the SR_AUTOTUNE_CACHE file."""
    import json
    from paper_2402_08725_gb300.binding import Batch, Problem
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("SR_AUTOTUNE_CACHE", str(cache))
    fd = syn.small_deconv(seed=91, E=6, N=44, f=2, K=19, M=1, J=3, lam=1.0)
    probs = [Problem.from_field(fd), Problem.from_field(fd, conv_mode="direct")]
    batch = Batch(probs)
    forms = batch.field_forms()
    assert forms[0] in ("direct", "fft") and forms[1] == "direct"
    data = json.loads(cache.read_text())
    assert data["44,2,19,1"] == (1 if forms[0] == "fft" else 0)
    P = torch.from_numpy(batch.pack([fd.params, fd.params])).cuda()
    losses = torch.empty(2, dtype=torch.float64, device="cuda")
    batch.loss_and_grad(P, losses=losses)
    l = losses.cpu().numpy()
    assert abs(l[0] - l[1]) <= 1e-6 * abs(l[1])
    batch.close()
    for p in probs:
        p.close()


def test_guard_bands_uneven_batch_both_forms(monkeypatch):
    """With guard tails on every device buffer, an uneven batch mixing both forms, several
    transform sizes and several epoch chunks per field writes nothing past any buffer, and
    each field still equals its single-problem evaluation."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    monkeypatch.setenv("SR_GUARD", "1")
    shapes = [(20, 32, "fft"), (9, 96, "fft"), (3, 48, "direct"), (17, 64, "fft"), (11, 128, "fft"),
              (5, 40, "direct")]
    fields = [syn.small_deconv(seed=300 + i, E=E, N=N, f=2, K=17, M=1, J=4, lam=1.0)
              for i, (E, N, _) in enumerate(shapes)]
    probs = [Problem.from_field(fd, conv_mode=m) for fd, (_, _, m) in zip(fields, shapes)]
    batch = Batch(probs)
    assert batch.field_forms() == [m for (_, _, m) in shapes]
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    total, grad = batch.loss_and_grad(P, losses=losses)
    for i, (fd, pr) in enumerate(zip(fields, probs)):
        l_i, g_i = pr.loss_and_grad(torch.from_numpy(fd.params).cuda())
        o = batch.offsets[i]
        assert losses[i].item() == l_i
        assert torch.equal(grad[o:o + fd.n_params], g_i)
    batch.close()
    for pr in probs:
        pr.close()


def test_schedules_forced_and_tuned_agree(tmp_path, monkeypatch):
    """Epochs per work item and the pair cap of the transform form change only the order of FP32
    sums (the pair cap changes which rows share an FP32 partial of chi^2): every forced schedule
    gives the losses within 1e-8 and the gradients within 1e-5 of each other, and the oracle's
    parity; the tuner keeps one of the candidates and caches it."""
    import json
    from paper_2402_08725_gb300.binding import Batch, Problem
    monkeypatch.setenv("SR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    fields = [syn.small_deconv(seed=970 + i, E=E, N=N, f=2, K=21, M=1, J=3, lam=1.0)
              for i, (E, N) in enumerate([(21, 48), (9, 64), (34, 32), (5, 96)])]
    probs = [Problem.from_field(fd, conv_mode="fft") for fd in fields]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in fields])).cuda()
    losses = torch.empty(len(fields), dtype=torch.float64, device="cuda")
    batch.set_schedule(16, 0)
    _, g_ref = batch.loss_and_grad(P, losses=losses)
    l_ref, g_ref = losses.cpu().numpy().copy(), g_ref.cpu().numpy().copy()
    for i, fd in enumerate(fields):
        o = batch.offsets[i]
        check_deconv(fd, float(l_ref[i]), g_ref[o:o + fd.n_params])
    from tests._helpers import rel_l2
    for c, g in [(2, 0), (4, 1), (8, 0), (16, 1), (6, 0)]:
        batch.set_schedule(c, g)
        assert batch.schedule() == (c, g)
        _, gr = batch.loss_and_grad(P, losses=losses)
        l = losses.cpu().numpy()
        assert np.all(np.abs(l - l_ref) <= 1e-8 * np.abs(l_ref)), (c, g, l, l_ref)
        assert rel_l2(gr.cpu().numpy(), g_ref) <= 1e-5, (c, g)
    t = batch.tune_schedule()
    assert t["epochs_per_item"] in (2, 4, 8, 16) and t["pairs_per_group"] in (0, 1) and t["ms_per_eval"] > 0
    assert batch.schedule() == (t["epochs_per_item"], t["pairs_per_group"])
    assert any(k.startswith("schedule:") for k in json.loads((tmp_path / "tune.json").read_text()))
    _, gr = batch.loss_and_grad(P, losses=losses)
    assert np.all(np.abs(losses.cpu().numpy() - l_ref) <= 1e-8 * np.abs(l_ref))
    batch.close()
    batch2 = Batch(probs)
    t2 = batch2.tune_schedule()   # the cached choice, not timed again
    assert t2["ms_per_eval"] is None
    assert (t2["epochs_per_item"], t2["pairs_per_group"]) == (t["epochs_per_item"], t["pairs_per_group"])
    with pytest.raises(Exception):
        batch2.set_schedule(3, 0)
    batch2.close()
    for pr in probs:
        pr.close()


# Starlet forms of wide fields: F = 420 (J = 5, 6) and F = 300 (J = 7) run as comb bands (rows
# rho + s k of one comb per block, the mirror preimages read from the plane); F = 720 is too wide
# for them and runs as comb tiles of 128 columns (the last tile column 80 wide) with J = 5, 7, 8.
@pytest.mark.parametrize("E,N,f,K,M,J", [(2, 140, 3, 15, 2, 5), (2, 140, 3, 15, 1, 6), (2, 150, 2, 9, 1, 7),
                                         (2, 240, 3, 9, 1, 5), (2, 240, 3, 9, 1, 7), (2, 240, 3, 9, 1, 8)])
def test_wide_field_starlet_forms_match_oracle(E, N, f, K, M, J):
    fd = syn.small_deconv(seed=3000 + N + J, E=E, N=N, f=f, K=K, M=M, J=J, lam=1.4, pos_half=N / 5)
    loss, g = _run(fd, conv_mode="direct")
    r = check_deconv(fd, loss, g)
    print("wide starlet", N, f, J, r)


def test_item_sums_alone_and_in_a_large_batch_bitwise():
    """A transform-form field of many work items (300 epochs: 19 items of 16) evaluated alone
    (few blocks: its items' accumulators are pre-summed, four lanes per spectral point) and inside
    a batch with enough transform fields to skip the pre-sum (each block sums its points itself)
    gives the same loss and gradient bit for bit: both take the items in the same 16-part order."""
    from paper_2402_08725_gb300.binding import Batch, Problem
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    big = syn.small_deconv(seed=611, E=300, N=16, f=2, K=9, M=1, J=3, lam=1.0)
    small = [syn.small_deconv(seed=620 + i, E=2, N=12, f=2, K=7, M=1, J=3, lam=1.0) for i in range(n_sms // 2 + 2)]
    single = Problem.from_field(big, conv_mode="fft")
    l1, g1 = single.loss_and_grad(torch.from_numpy(big.params).cuda())
    g1 = g1.clone()
    check_deconv(big, l1, g1.cpu().numpy())
    probs = [Problem.from_field(fd, conv_mode="fft") for fd in [big] + small]
    batch = Batch(probs)
    P = torch.from_numpy(batch.pack([fd.params for fd in [big] + small])).cuda()
    losses = torch.empty(len(probs), dtype=torch.float64, device="cuda")
    _, grad = batch.loss_and_grad(P, losses=losses)
    assert losses[0].item() == l1
    assert torch.equal(grad[:big.n_params], g1)
    batch.close()
    for q in probs + [single]:
        q.close()
