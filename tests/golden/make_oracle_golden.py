"""Writes oracle_small_cases.txt: loss and per-block gradient norms of small seeded cases,
computed by the FP64 oracle only (regression values for the oracle; no GPU, no library), and
oracle_small_cases_inputs.txt: the float32 inputs of those cases (data, sigma, PSFs, weights,
parameters), so that the stored values are reproduced from the very same inputs on every
machine, whatever the last bits of the seeded generator there.

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


ARRAYS = ("d", "sigma", "s", "W", "params")
INPUTS = os.path.join(HERE, "oracle_small_cases_inputs.txt")


def generated_inputs():
    """{case: {array: float32 array}} from the seeded generator (used when writing)."""
    out = {}
    for name, seed, E, N, f, K, M, J, lam, lp in CASES:
        fd = syn.small_deconv(seed, E=E, N=N, f=f, K=K, M=M, J=J, lam=lam)
        out[name] = {a: np.asarray(getattr(fd, a), dtype=np.float32) for a in ARRAYS}
    return out


def stored_inputs():
    """{case: {array: float32 array}} read back from oracle_small_cases_inputs.txt."""
    out = {}
    for line in open(INPUTS):
        if line.startswith("#"):
            continue
        t = line.split()
        name, arr, ndim = t[0], t[1], int(t[2])
        shape = tuple(int(v) for v in t[3:3 + ndim])
        vals = np.array([float(v) for v in t[3 + ndim:]], dtype=np.float32)
        out.setdefault(name, {})[arr] = vals.reshape(shape)
    return out


def rows(inputs=None):
    """Oracle values of every case, on the given inputs (default: the stored ones)."""
    inputs = stored_inputs() if inputs is None else inputs
    out = []
    for name, seed, E, N, f, K, M, J, lam, lp in CASES:
        fd = syn.small_deconv(seed, E=E, N=N, f=f, K=K, M=M, J=J, lam=lam)
        for a in ARRAYS:
            setattr(fd, a, inputs[name][a])
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
    gen = generated_inputs()
    with open(INPUTS, "w") as fh:
        fh.write("# Written by tests/golden/make_oracle_golden.py: float32 inputs of its cases, one array per line:\n")
        fh.write("# case, array, ndim, shape, values (9 significant digits: exact float32 round trip)\n")
        for name, arrs in gen.items():
            for a in ARRAYS:
                v = arrs[a]
                fh.write(f"{name} {a} {v.ndim} " + " ".join(str(n) for n in v.shape) + " " +
                         " ".join(f"{x:.9g}" for x in v.ravel()) + "\n")
    assert all(np.array_equal(stored_inputs()[n][a], gen[n][a]) for n in gen for a in ARRAYS)
    with open(os.path.join(HERE, "oracle_small_cases.txt"), "w") as fh:
        fh.write("# Written by tests/golden/make_oracle_golden.py from the FP64 oracle (small_deconv cases of\n")
        fh.write("# that script, lambda_pts as listed there): case, loss, gradient L2 norm per block (h a c delta Gamma)\n")
        for name, L, norms in rows():
            fh.write(f"{name} {L:.15e} " + " ".join(f"{v:.15e}" for v in norms) + "\n")
