"""Writes oracle_small_cases.txt: loss and per-block gradient norms of small seeded cases,
computed by the FP64 oracle only (regression values for the oracle; no GPU, no library).

    python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2402_08725_gb300 import synthetic as syn  # noqa: E402

CASES = [  # (name, seed, E, N, f, K, M, J, lam, lam_pts)
    ("deconv_a", 101, 3, 16, 2, 13, 2, 3, 1.0, 0.0),
    ("deconv_b", 102, 2, 20, 2, 9, 1, 4, 0.5, 0.7),
    ("deconv_c", 103, 4, 12, 3, 7, 0, 3, 2.0, 0.0),
]
BLOCKS = ("h", "a", "c", "delta", "Gamma")


def rows():
    out = []
    for name, seed, E, N, f, K, M, J, lam, lp in CASES:
        fd = syn.small_deconv(seed, E=E, N=N, f=f, K=K, M=M, J=J, lam=lam)
        P = fd.params.astype(np.float64)
        L, _, g, _ = oracle.deconv_loss_grad(fd.E, fd.N, fd.f, fd.K, fd.M, fd.J, fd.lam, fd.d, fd.sigma, fd.s,
                                             fd.W, P)
        if lp > 0:
            v, gp = oracle.pts_prior(fd.E, fd.N, fd.f, fd.M, fd.J, lp, fd.W, P)
            L, g = L + v, g + gp
        F = f * N
        sizes = [F * F, E * M, 2 * M, 2 * E, E]
        o, norms = 0, []
        for n in sizes:
            norms.append(float(np.linalg.norm(g[o:o + n])))
            o += n
        out.append((name, L, norms))
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small_cases.txt"), "w") as fh:
        fh.write("# Written by tests/golden/make_oracle_golden.py from the FP64 oracle (small_deconv cases of\n")
        fh.write("# that script, lambda_pts as listed there): case, loss, gradient L2 norm per block (h a c delta Gamma)\n")
        for name, L, norms in rows():
            fh.write(f"{name} {L:.15e} " + " ".join(f"{v:.15e}" for v in norms) + "\n")
