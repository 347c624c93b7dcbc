"""Python front end of the C ABI: Problem and Batch objects over torch device memory.

Every computation happens in the CUDA library; this module converts torch
tensors and numpy arrays into pointers and sizes and passes the caller's
current CUDA stream.  Parameter vectors follow the packed layouts of
include/starred.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as nat


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _as_input(x, n_expected: int):
    """(pointer, on_device, keepalive) for a float32 array given as a CUDA tensor,
    CPU tensor or numpy array."""
    if isinstance(x, torch.Tensor):
        t = x.detach()
        if t.dtype != torch.float32:
            t = t.float()
        t = t.contiguous()
        if t.numel() != n_expected:
            raise ValueError(f"expected {n_expected} values, got {t.numel()}")
        return ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, t
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if a.size != n_expected:
        raise ValueError(f"expected {n_expected} values, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data), 0, a


def _check_host_arrays(specs):
    for a, n, dt, name in specs:
        if not isinstance(a, np.ndarray) or a.dtype != dt or a.size < n or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name} must be a contiguous {np.dtype(dt).name} array of {n} values")


def _cuda_f32(t: torch.Tensor, n: int, name: str):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} values, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def optim_cfg(kind="adabelief", lr=(1e-2,), beta1=0.9, beta2=0.999, eps=None) -> nat.OptimCfg:
    k = nat.SR_ADABELIEF if kind == "adabelief" else nat.SR_ADAM
    if eps is None:
        eps = 1e-16 if k == nat.SR_ADABELIEF else 1e-8
    cfg = nat.OptimCfg()
    cfg.kind = k
    cfg.beta1, cfg.beta2, cfg.eps = beta1, beta2, eps
    lrs = list(lr) + [0.0] * (nat.SR_MAX_GROUPS - len(lr))
    for i in range(nat.SR_MAX_GROUPS):
        cfg.lr[i] = float(lrs[i])
    return cfg


class Problem:
    """One STARRED problem (a deconvolution field, or a PSF fit) on the current GPU."""

    def __init__(self, kind: str, E: int, N: int, f: int, K: int = 1, M: int = 0, J: int = 4, lam: float = 0.0,
                 conv_mode: str = "auto", stream=None):
        self.lib = nat.load()
        self.kind = nat.SR_DECONV if kind == "deconv" else nat.SR_PSF
        self.E, self.N, self.f, self.K, self.M, self.J, self.lam = E, N, f, K, M, J, lam
        d = nat.ProblemDesc()
        d.kind, d.n_epochs, d.data_n, d.supersampling = self.kind, E, N, f
        d.psf_k, d.n_sources, d.n_scales, d.lam = K, M, J, lam
        d.conv_mode = {"auto": nat.SR_CONV_AUTO, "direct": nat.SR_CONV_DIRECT, "plain": nat.SR_CONV_PLAIN,
                       "fft": nat.SR_CONV_FFT}[conv_mode]
        self._stream = stream
        h = ctypes.c_void_p()
        nat.check(self.lib.sr_create_problem(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)), "sr_create_problem")
        self.handle = h
        self.n_params = int(self.lib.sr_param_count(h))
        self._grad = None
        self._loss_dev = None

    @classmethod
    def from_field(cls, fd, conv_mode="auto", stream=None, data=True):
        """Problem for a synthetic.DeconvField (data, noise, PSFs and weights set)."""
        p = cls("deconv", fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, conv_mode=conv_mode, stream=stream)
        if data:
            p.set_data(fd.d)
            p.set_noise(fd.sigma)
            p.set_psfs(fd.s)
            p.set_weights(fd.W)
        return p

    @classmethod
    def from_psf(cls, pb, stream=None):
        p = cls("psf", pb.S, pb.N, pb.f, J=pb.J, lam=pb.lam, stream=stream)
        p.set_data(pb.t)
        p.set_noise(pb.sigma)
        p.set_weights(pb.W)
        return p

    # --- inputs -------------------------------------------------------------------------
    def set_data(self, x):
        ptr, dev, keep = _as_input(x, self.E * self.N * self.N)
        nat.check(self.lib.sr_set_data(self.handle, ptr, dev), "sr_set_data")
        self._keep_d = keep

    def set_noise(self, x):
        ptr, dev, keep = _as_input(x, self.E * self.N * self.N)
        nat.check(self.lib.sr_set_noise(self.handle, ptr, dev), "sr_set_noise")
        self._keep_s = keep

    def set_psfs(self, x):
        ptr, dev, keep = _as_input(x, self.E * self.K * self.K)
        nat.check(self.lib.sr_set_psfs(self.handle, ptr, dev), "sr_set_psfs")
        self._keep_p = keep

    def set_weights(self, W):
        a = np.ascontiguousarray(np.asarray(W, dtype=np.float32))
        if a.size != self.J - 1:
            raise ValueError(f"expected {self.J - 1} weights")
        nat.check(self.lib.sr_set_weights(self.handle, ctypes.c_void_p(a.ctypes.data)), "sr_set_weights")

    def set_weight_map(self, Wmap=None):
        """Prior weights per starlet coefficient, [J-1][F][F] (numpy or a CUDA tensor), or None to
        go back to the per-scale weights; sr_set_weight_map."""
        if Wmap is None:
            nat.check(self.lib.sr_set_weight_map(self.handle, None, 0), "sr_set_weight_map")
            return
        F = self.f * self.N
        ptr, dev, keep = _as_input(Wmap, (self.J - 1) * F * F)
        nat.check(self.lib.sr_set_weight_map(self.handle, ptr, dev), "sr_set_weight_map")
        del keep

    def set_lambda_pts(self, lambda_pts: float):
        """Strength of the point-source prior (Eq. 11, third term); sr_set_lambda_pts."""
        nat.check(self.lib.sr_set_lambda_pts(self.handle, float(lambda_pts)), "sr_set_lambda_pts")

    def set_translate_h(self, enable: bool = True):
        """Move the extended channel with each epoch's shift (sec. 5; bilinear, zero outside);
        sr_set_translate_h.  Direct form only; drops the problem's plan and optimiser state."""
        nat.check(self.lib.sr_set_translate_h(self.handle, 1 if enable else 0), "sr_set_translate_h")

    def set_rotations(self, theta=None):
        """Rotate each epoch's frame by theta[i] radians about the grid centre (sec. 5), or None
        to turn the rotations off; sr_set_rotations.  Direct form only."""
        if theta is None:
            nat.check(self.lib.sr_set_rotations(self.handle, None), "sr_set_rotations")
            return
        a = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if a.size != self.E:
            raise ValueError(f"expected {self.E} angles")
        nat.check(self.lib.sr_set_rotations(self.handle, a.ctypes.data_as(nat.P_double)), "sr_set_rotations")

    def estimate_lambda_pts(self, params: torch.Tensor) -> float:
        """lambda_pts from the model `params` by the ratio of App. C; sr_estimate_lambda_pts."""
        out = ctypes.c_double()
        nat.check(self.lib.sr_estimate_lambda_pts(self.handle, _cuda_f32(params, self.n_params, "params"),
                                                  ctypes.byref(out)), "sr_estimate_lambda_pts")
        return float(out.value)

    def layout(self):
        L = nat.Layout()
        nat.check(self.lib.sr_param_layout(self.handle, ctypes.byref(L)), "sr_param_layout")
        return [(int(L.offset[g]), int(L.count[g])) for g in range(L.n_groups)]

    # --- evaluation ------------------------------------------------------------------------
    def loss_and_grad(self, params: torch.Tensor, grad: torch.Tensor | None = None, sync: bool = True):
        """Returns (loss, grad).  loss is a float when sync, else a 0-d float64 CUDA tensor."""
        if grad is None:
            grad = torch.empty(self.n_params, dtype=torch.float32, device=params.device)
        pp = _cuda_f32(params, self.n_params, "params")
        gp = _cuda_f32(grad, self.n_params, "grad")
        if sync:
            loss = ctypes.c_double()
            nat.check(self.lib.sr_loss_and_grad(self.handle, pp, ctypes.byref(loss), None, gp), "sr_loss_and_grad")
            return loss.value, grad
        loss_t = torch.empty((), dtype=torch.float64, device=params.device)
        nat.check(self.lib.sr_loss_and_grad(self.handle, pp, None, ctypes.c_void_p(loss_t.data_ptr()), gp),
                  "sr_loss_and_grad")
        return loss_t, grad

    def loss(self, params: torch.Tensor) -> float:
        loss = ctypes.c_double()
        nat.check(self.lib.sr_loss(self.handle, _cuda_f32(params, self.n_params, "params"), ctypes.byref(loss)), "sr_loss")
        return loss.value

    def loss_and_grad_host(self, params_host: np.ndarray, grad_host: np.ndarray | None = None):
        p = np.ascontiguousarray(params_host, dtype=np.float32)
        if grad_host is None:
            grad_host = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        nat.check(self.lib.sr_loss_and_grad_host(self.handle, ctypes.c_void_p(p.ctypes.data), ctypes.byref(loss),
                                                 ctypes.c_void_p(grad_host.ctypes.data)), "sr_loss_and_grad_host")
        return loss.value, grad_host

    def loss_and_grad_host_async(self, params_host, grad_host, loss_host):
        """Queue the host-buffer evaluation without waiting (sr_loss_and_grad_host_async).
        params_host, grad_host (n_params float32) and loss_host (one float64) are host arrays,
        page-locked for the call to return at once; they are read or written until sync()."""
        _check_host_arrays(((params_host, self.n_params, np.float32, "params_host"),
                            (grad_host, self.n_params, np.float32, "grad_host"),
                            (loss_host, 1, np.float64, "loss_host")))
        nat.check(self.lib.sr_loss_and_grad_host_async(self.handle, ctypes.c_void_p(params_host.ctypes.data),
                                                       ctypes.c_void_p(loss_host.ctypes.data),
                                                       ctypes.c_void_p(grad_host.ctypes.data)),
                  "sr_loss_and_grad_host_async")

    def sync(self):
        """Wait for the problem's stream and raise on the set-up's input checks (sr_sync)."""
        nat.check(self.lib.sr_sync(self.handle), "sr_sync")

    def step(self, params: torch.Tensor, n_steps: int, cfg: nat.OptimCfg, losses: torch.Tensor | None = None,
             sync: bool = True) -> float | None:
        """n_steps optimiser updates in place (sr_step).  Returns the last loss, read back with a
        synchronisation of the problem's stream; with sync=False nothing is read back (None) and
        the call returns once the steps are queued."""
        last = ctypes.c_double()
        lp = None
        if losses is not None:
            if losses.dtype != torch.float64 or not losses.is_cuda or losses.numel() < n_steps:
                raise TypeError("losses must be a float64 CUDA tensor with n_steps values")
            lp = ctypes.c_void_p(losses.data_ptr())
        nat.check(self.lib.sr_step(self.handle, _cuda_f32(params, self.n_params, "params"), int(n_steps),
                                   ctypes.byref(cfg), lp, ctypes.byref(last) if sync else None), "sr_step")
        return last.value if sync else None

    def psf_model(self, params: torch.Tensor) -> torch.Tensor:
        """The narrow PSF s = Moffat + b of a PSF fit's parameters, [F][F] on the device; sr_psf_model."""
        F = self.f * self.N
        out = torch.empty((F, F), dtype=torch.float32, device=params.device)
        nat.check(self.lib.sr_psf_model(self.handle, _cuda_f32(params, self.n_params, "params"),
                                        ctypes.c_void_p(out.data_ptr())), "sr_psf_model")
        return out

    def lbfgsb(self, params: torch.Tensor, max_iter: int = 100, m: int = 10, max_ls: int = 20, pgtol: float = 1e-5,
               factr: float = 1e7):
        """L-BFGS-B from `params` (overwritten); sr_lbfgsb.  Returns a dict: iterations,
        evaluations, status, f, pg_norm and the loss history (start and every iterate)."""
        cfg = nat.LbfgsbCfg(int(m), int(max_iter), int(max_ls), float(pgtol), float(factr))
        info = nat.LbfgsbInfo()
        hist = np.zeros(int(max_iter) + 1)
        nat.check(self.lib.sr_lbfgsb(self.handle, _cuda_f32(params, self.n_params, "params"), ctypes.byref(cfg),
                                     hist.ctypes.data_as(nat.P_double), ctypes.byref(info)), "sr_lbfgsb")
        return {"iterations": info.iterations, "evaluations": info.evaluations,
                "status": nat.LBFGSB_STATUS.get(info.status, str(info.status)), "f": info.f, "pg_norm": info.pg_norm,
                "history": hist[:info.iterations + 1]}

    def reset_optimizer(self):
        nat.check(self.lib.sr_reset_optimizer(self.handle), "sr_reset_optimizer")

    def get_state(self):
        m = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        v = torch.empty_like(m)
        t = ctypes.c_int64()
        nat.check(self.lib.sr_get_state(self.handle, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                        ctypes.byref(t)), "sr_get_state")
        return m, v, t.value

    def set_state(self, m: torch.Tensor, v: torch.Tensor, t: int):
        nat.check(self.lib.sr_set_state(self.handle, _cuda_f32(m, self.n_params, "m"), _cuda_f32(v, self.n_params, "v"),
                                        int(t)), "sr_set_state")

    def launches_per_eval(self) -> int:
        return int(self.lib.sr_launches_per_eval(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many deconvolution fields evaluated together (one launch per kernel for all fields)."""

    def __init__(self, problems, stream=None):
        self.lib = nat.load()
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle for p in self.problems])
        h = ctypes.c_void_p()
        nat.check(self.lib.sr_batch_create(arr, len(self.problems), _stream_ptr(stream), ctypes.byref(h)),
                  "sr_batch_create")
        self.handle = h
        self.n_params = int(self.lib.sr_batch_param_count(h))
        self.offsets = []
        for i in range(len(self.problems)):
            o = ctypes.c_size_t()
            nat.check(self.lib.sr_batch_param_offset(h, i, ctypes.byref(o)), "sr_batch_param_offset")
            self.offsets.append(int(o.value))

    def _set(self, fn, name, x):
        if isinstance(x, torch.Tensor):
            t = x.detach().float().contiguous()
            nat.check(fn(self.handle, ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0), name)
            return t
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
        nat.check(fn(self.handle, ctypes.c_void_p(a.ctypes.data), 0), name)
        return a

    def set_data(self, d):
        """Every member's data, concatenated in batch order (sr_batch_set_data)."""
        return self._set(self.lib.sr_batch_set_data, "sr_batch_set_data", d)

    def set_noise(self, sigma):
        return self._set(self.lib.sr_batch_set_noise, "sr_batch_set_noise", sigma)

    def set_psfs(self, s):
        return self._set(self.lib.sr_batch_set_psfs, "sr_batch_set_psfs", s)

    def pack(self, vectors):
        """Concatenate per-field parameter vectors (numpy or torch) in batch order."""
        if isinstance(vectors[0], torch.Tensor):
            return torch.cat([v.reshape(-1).float() for v in vectors])
        return np.concatenate([np.asarray(v, dtype=np.float32).ravel() for v in vectors])

    def loss_and_grad(self, params: torch.Tensor, grad: torch.Tensor | None = None, losses: torch.Tensor | None = None,
                      sync: bool = True):
        if grad is None:
            grad = torch.empty(self.n_params, dtype=torch.float32, device=params.device)
        lp = None
        if losses is not None:
            lp = ctypes.c_void_p(losses.data_ptr())
        pp = _cuda_f32(params, self.n_params, "params")
        gp = _cuda_f32(grad, self.n_params, "grad")
        if sync:
            tot = ctypes.c_double()
            nat.check(self.lib.sr_batch_loss_and_grad(self.handle, pp, lp, None, ctypes.byref(tot), gp),
                      "sr_batch_loss_and_grad")
            return tot.value, grad
        tot_t = torch.empty((), dtype=torch.float64, device=params.device)
        nat.check(self.lib.sr_batch_loss_and_grad(self.handle, pp, lp, ctypes.c_void_p(tot_t.data_ptr()), None, gp),
                  "sr_batch_loss_and_grad")
        return tot_t, grad

    def loss_and_grad_host(self, params_host: np.ndarray, grad_host: np.ndarray | None = None):
        p = np.ascontiguousarray(params_host, dtype=np.float32)
        if grad_host is None:
            grad_host = np.empty(self.n_params, dtype=np.float32)
        tot = ctypes.c_double()
        nat.check(self.lib.sr_batch_loss_and_grad_host(self.handle, ctypes.c_void_p(p.ctypes.data), ctypes.byref(tot),
                                                       ctypes.c_void_p(grad_host.ctypes.data)),
                  "sr_batch_loss_and_grad_host")
        return tot.value, grad_host

    def loss_and_grad_host_async(self, params_host, grad_host, total_host):
        """Queue the host-buffer evaluation without waiting (sr_batch_loss_and_grad_host_async).
        params_host, grad_host (n_params float32) and total_host (one float64) are host arrays,
        page-locked for the call to return at once (numpy views of pinned torch tensors); they are
        written or read until sync()."""
        _check_host_arrays(((params_host, self.n_params, np.float32, "params_host"),
                            (grad_host, self.n_params, np.float32, "grad_host"),
                            (total_host, 1, np.float64, "total_host")))
        nat.check(self.lib.sr_batch_loss_and_grad_host_async(self.handle, ctypes.c_void_p(params_host.ctypes.data),
                                                             ctypes.c_void_p(total_host.ctypes.data),
                                                             ctypes.c_void_p(grad_host.ctypes.data)),
                  "sr_batch_loss_and_grad_host_async")

    def sync(self):
        """Wait for the batch's stream and raise on the queued set-up's input checks (sr_batch_sync)."""
        nat.check(self.lib.sr_batch_sync(self.handle), "sr_batch_sync")

    def step(self, params: torch.Tensor, n_steps: int, cfg: nat.OptimCfg, sync: bool = True) -> float | None:
        """n_steps optimiser updates of every field (sr_batch_step).  Returns the last total loss
        (synchronises the batch's stream), or None without reading it back when sync=False."""
        last = ctypes.c_double()
        nat.check(self.lib.sr_batch_step(self.handle, _cuda_f32(params, self.n_params, "params"), int(n_steps),
                                         ctypes.byref(cfg), ctypes.byref(last) if sync else None), "sr_batch_step")
        return last.value if sync else None

    def lbfgsb(self, params: torch.Tensor, max_iter: int = 100, m: int = 10, max_ls: int = 20, pgtol: float = 1e-5,
               factr: float = 1e7):
        """L-BFGS-B on the batch's total loss from `params` (overwritten); sr_batch_lbfgsb."""
        cfg = nat.LbfgsbCfg(int(m), int(max_iter), int(max_ls), float(pgtol), float(factr))
        info = nat.LbfgsbInfo()
        hist = np.zeros(int(max_iter) + 1)
        nat.check(self.lib.sr_batch_lbfgsb(self.handle, _cuda_f32(params, self.n_params, "params"), ctypes.byref(cfg),
                                           hist.ctypes.data_as(nat.P_double), ctypes.byref(info)), "sr_batch_lbfgsb")
        return {"iterations": info.iterations, "evaluations": info.evaluations,
                "status": nat.LBFGSB_STATUS.get(info.status, str(info.status)), "f": info.f, "pg_norm": info.pg_norm,
                "history": hist[:info.iterations + 1]}

    def lbfgsb_fields(self, params: torch.Tensor, max_iter: int = 100, m: int = 10, max_ls: int = 20,
                      pgtol: float = 1e-5, factr: float = 1e7):
        """One L-BFGS-B run per field from `params` (overwritten); sr_batch_lbfgsb_fields.  Returns
        (a dict per field: iterations, evaluations, status, f, pg_norm, history; the number of
        batched evaluations after the first)."""
        cfg = nat.LbfgsbCfg(int(m), int(max_iter), int(max_ls), float(pgtol), float(factr))
        nf = len(self.problems)
        infos = (nat.LbfgsbInfo * nf)()
        hist = np.zeros((nf, int(max_iter) + 1))
        rounds = ctypes.c_int()
        nat.check(self.lib.sr_batch_lbfgsb_fields(self.handle, _cuda_f32(params, self.n_params, "params"),
                                                  ctypes.byref(cfg), hist.ctypes.data_as(nat.P_double), infos,
                                                  ctypes.byref(rounds)), "sr_batch_lbfgsb_fields")
        out = []
        for f in range(nf):
            info = infos[f]
            out.append({"iterations": info.iterations, "evaluations": info.evaluations,
                        "status": nat.LBFGSB_STATUS.get(info.status, str(info.status)), "f": info.f,
                        "pg_norm": info.pg_norm, "history": hist[f, :info.iterations + 1].copy()})
        return out, rounds.value

    def reset_optimizer(self):
        nat.check(self.lib.sr_batch_reset_optimizer(self.handle), "sr_batch_reset_optimizer")

    def launches_per_eval(self) -> int:
        return int(self.lib.sr_batch_launches_per_eval(self.handle))

    def field_forms(self):
        """'direct' or 'fft' for each field, as chosen when the batch was created."""
        return ["fft" if self.lib.sr_batch_field_form(self.handle, i) == nat.SR_CONV_FFT else "direct"
                for i in range(len(self.problems))]

    def set_schedule(self, epochs_per_item: int = 0, pairs_per_group: int = 0):
        """Schedule of the transform form (0 = automatic); rebuilds the batch's plan."""
        nat.check(self.lib.sr_batch_set_schedule(self.handle, int(epochs_per_item), int(pairs_per_group)),
                  "sr_batch_set_schedule")

    def schedule(self):
        """(epochs per work item, pair cap) of the plan in use."""
        c, g = ctypes.c_int(), ctypes.c_int()
        nat.check(self.lib.sr_batch_get_schedule(self.handle, ctypes.byref(c), ctypes.byref(g)),
                  "sr_batch_get_schedule")
        return c.value, g.value

    def tune_schedule(self):
        """Times the candidate schedules and keeps the fastest (or the cached choice):
        {"epochs_per_item", "pairs_per_group", "ms_per_eval" (None when cached)}."""
        c, g, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        nat.check(self.lib.sr_batch_tune_schedule(self.handle, ctypes.byref(c), ctypes.byref(g), ctypes.byref(ms)),
                  "sr_batch_tune_schedule")
        return {"epochs_per_item": c.value, "pairs_per_group": g.value,
                "ms_per_eval": None if ms.value < 0 else float(ms.value)}

    def profile(self, enable: bool = True):
        nat.check(self.lib.sr_batch_profile(self.handle, 1 if enable else 0), "sr_batch_profile")

    def profile_read(self):
        """(evaluations recorded, summed ms of the forward tile kernel, of the adjoint tile
        kernel, and of the transform kernels)."""
        n, fm, am, tm = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        nat.check(self.lib.sr_batch_profile_read(self.handle, ctypes.byref(n), ctypes.byref(fm), ctypes.byref(am),
                                                 ctypes.byref(tm)), "sr_batch_profile_read")
        return n.value, fm.value, am.value, tm.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak() -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s (sr_measure_fp32_peak)."""
    lib = nat.load()
    t = ctypes.c_double()
    nat.check(lib.sr_measure_fp32_peak(ctypes.byref(t)), "sr_measure_fp32_peak")
    return float(t.value)


def noise_weights(N: int, f: int, K: int, J: int, sigma: torch.Tensor, s1: torch.Tensor, n_real: int, seed: int,
                  want_map: bool = True, timing: bool = False, stream=None):
    """Monte Carlo prior weights of sec. 2.3 (sr_noise_weights) from sigma [E][N][N] and the
    narrow PSF s1 [K][K], both float32 CUDA tensors.  Returns (W_scale as a numpy float32 [J-1],
    W_map as a CUDA tensor [J-1][fN][fN] or None, the phase timings as a dict or None)."""
    lib = nat.load()
    E = sigma.numel() // (N * N)
    sp = _cuda_f32(sigma, E * N * N, "sigma")
    kp = _cuda_f32(s1, K * K, "s1")
    F = f * N
    W = np.zeros(J - 1, dtype=np.float32)
    W_map = torch.empty((J - 1, F, F), dtype=torch.float32, device=sigma.device) if want_map else None
    tm = nat.NoiseTiming() if timing else None
    nat.check(lib.sr_noise_weights(N, f, K, J, E, sp, kp, int(n_real), ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                   W.ctypes.data_as(nat.P_float),
                                   ctypes.c_void_p(W_map.data_ptr()) if W_map is not None else None,
                                   ctypes.byref(tm) if tm is not None else None, _stream_ptr(stream)),
              "sr_noise_weights")
    times = None
    if tm is not None:
        times = {k: getattr(tm, k) for k, _ in nat.NoiseTiming._fields_}
    return W, W_map, times
