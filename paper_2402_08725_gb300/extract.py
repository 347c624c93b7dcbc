"""End-to-end light-curve extraction of one field (sec. 3): a data-driven starting point, the
optimiser through the library's captured steps (sec. 2.4: AdaBelief), the point-source prior
with its App. C refinement, and the estimated light curves and positions read back.

Starting point: the extended source h = the per-pixel median of the data over the epochs with
the (2r+1)^2 data-pixel box around each catalogue position c0_k replaced by the median of the
ring of width 3 around the box (the point sources taken out), each data pixel spread evenly over
its f x f fine pixels; c = c0 (data pixels from the stamp centre); a_ki = the flux of d_i minus
that extended image in the box around c0_k, clipped at 0; delta = 0; Gamma = 0.  Learning rates
per parameter group (h, a, c, delta, Gamma): 0.1 % of the brightest data pixel spread over f^2
fine pixels, 1 % of the mean starting amplitude, and fixed steps of 5e-3, 2e-3 and 1e-2.

The optimiser is AdaBelief with these rates, or L-BFGS-B (sr_lbfgsb, no rates), which may stop
before its iteration budget when its line search finds no step.

Point-source prior (App. C): lambda_pts starts at 0.5 lambda; the steps run in rounds, and after
each round lambda_pts is re-estimated from the current model (sr_estimate_lambda_pts, clipped at
0).  lambda_pts = a number fixes it instead; 0 leaves the term out.
"""
from __future__ import annotations

import numpy as np
import torch

from . import synthetic as syn
from .binding import Problem, optim_cfg


def initial_params(fd, c0, box: int = 3) -> np.ndarray:
    E, N, f, M = fd.E, fd.N, fd.f, fd.M
    c0 = np.asarray(c0, dtype=np.float64).reshape(M, 2)
    ext = np.median(fd.d.astype(np.float64), axis=0)
    centre = (N - 1) / 2.0
    boxes = []
    for k in range(M):
        x, y = int(round(centre + c0[k, 0])), int(round(centre + c0[k, 1]))
        boxes.append((slice(max(y - box, 0), min(y + box + 1, N)), slice(max(x - box, 0), min(x + box + 1, N))))
        ring = np.zeros((N, N), dtype=bool)
        ring[max(y - box - 3, 0):min(y + box + 4, N), max(x - box - 3, 0):min(x + box + 4, N)] = True
        ring[boxes[-1]] = False
        if ring.any():
            ext[boxes[-1]] = np.median(ext[ring])
    h0 = np.kron(ext, np.ones((f, f))) / (f * f)
    a0 = np.zeros((E, M))
    for i in range(E):
        d = fd.d[i].astype(np.float64) - ext
        for k in range(M):
            a0[i, k] = max(float(np.sum(d[boxes[k]])), 0.0)
    return syn.pack_deconv(h0, a0, c0, np.zeros((E, 2)), np.zeros(E))


def default_lr(fd, p0):
    E, M, f = fd.E, fd.M, fd.f
    F = f * fd.N
    a0 = p0[F * F:F * F + E * M]
    return (1e-3 * float(np.max(fd.d)) / (f * f), 1e-2 * max(float(np.mean(np.abs(a0))), 1.0), 5e-3, 2e-3, 1e-2)


def extract(fd, c0, n_steps: int = 200, lr=None, lambda_pts="app_c", rounds: int = 4, stream=None,
            optimizer: str = "adabelief"):
    """Run n_steps optimiser steps (AdaBelief; or L-BFGS-B iterations with optimizer="lbfgsb")
    from initial_params(fd, c0), in `rounds` rounds when lambda_pts is refined.  Returns a dict
    with the final packed parameters, the light curves a [E][M], the positions c [M][2], the loss
    of every step, the lambda_pts of each round and the device time of the steps and estimates
    (CUDA events on the problem's stream, ms); for L-BFGS-B also its loss evaluations."""
    prob = Problem.from_field(fd, stream=stream)
    p0 = initial_params(fd, c0)
    P = torch.from_numpy(np.ascontiguousarray(p0, dtype=np.float32)).cuda()
    cfg = optim_cfg("adabelief", lr=lr if lr is not None else default_lr(fd, p0))
    refine = lambda_pts == "app_c" and fd.M > 0
    lp = 0.5 * fd.lam if refine else float(lambda_pts)
    if lp > 0.0:
        prob.set_lambda_pts(lp)
    n_rounds = max(1, rounds) if refine else 1
    losses = torch.empty(max(n_steps, 1), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lps, done = [lp], 0
    e0.record(st)
    evals, hist = 0, []
    for r in range(n_rounds):
        n = (n_steps * (r + 1)) // n_rounds - done
        if n > 0:
            if optimizer == "lbfgsb":
                info = prob.lbfgsb(P, max_iter=n, pgtol=0.0, factr=0.0)
                evals += info["evaluations"]
                hist.extend(info["history"][1:])
            else:
                prob.step(P, n, cfg, losses[done:done + n])
            done += n
        if refine and r + 1 < n_rounds:
            lp = max(prob.estimate_lambda_pts(P), 0.0)
            prob.set_lambda_pts(lp)
            lps.append(lp)
    e1.record(st)
    e1.synchronize()
    out = P.cpu().numpy().astype(np.float64)
    _, a, c, _, _ = syn.unpack_deconv(out, fd.E, fd.N, fd.f, fd.M)
    L = np.asarray(hist) if optimizer == "lbfgsb" else losses[:n_steps].cpu().numpy()
    res = {"params": out, "a": a, "c": c, "losses": L, "lambda_pts": lps, "ms": e0.elapsed_time(e1),
           "evaluations": evals if optimizer == "lbfgsb" else n_steps}
    prob.close()
    return res
