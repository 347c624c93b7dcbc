"""Host-side checks of the C-ABI library (no GPU needed).

The library builds for sm_103a, loads, exports every function that
include/starred.h declares, and rejects invalid problem descriptions before
touching the device.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2402_08725_gb300 import _native as nat
from paper_2402_08725_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "starred.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(sr_[a-z0-9_]+)\s*\(", txt))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return nat.load(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(nat.PROTOTYPES)


def test_built_for_sm103(lib):
    assert lib.sr_build_arch() == 103
    assert lib.sr_version() >= 1


def _desc(**kw):
    d = nat.ProblemDesc()
    d.kind, d.n_epochs, d.data_n, d.supersampling = nat.SR_DECONV, 2, 16, 2
    d.psf_k, d.n_sources, d.n_scales, d.lam, d.conv_mode = 9, 1, 3, 1.0, 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,code", [
    ({"n_epochs": 0}, 2), ({"data_n": 0}, 2), ({"supersampling": 0}, 2), ({"n_scales": 1}, 2),
    ({"n_scales": 9}, 2), ({"data_n": 4, "supersampling": 1, "n_scales": 4}, 2), ({"psf_k": 0}, 2),
    ({"n_sources": -1}, 2), ({"lam": -1.0}, 1), ({"lam": float("nan")}, 1), ({"kind": 7}, 1),
    ({"conv_mode": 9}, 1), ({"kind": nat.SR_PSF, "conv_mode": nat.SR_CONV_PLAIN}, 8),
])
def test_invalid_descriptions_rejected_before_device_use(lib, kw, code):
    h = ctypes.c_void_p()
    rc = lib.sr_create_problem(ctypes.byref(_desc(**kw)), None, ctypes.byref(h))
    assert rc == code
    assert h.value is None
    assert lib.sr_last_error()


def test_null_arguments(lib):
    assert lib.sr_create_problem(None, None, None) == 1
    assert lib.sr_destroy(None) == 0
    assert lib.sr_batch_destroy(None) == 0
    assert lib.sr_param_count(None) == 0
    assert lib.sr_set_data(None, None, 0) == 1
    assert lib.sr_loss_and_grad(None, None, None, None, None) == 1


def test_batch_size_checked_before_its_members(lib):
    """sr_batch_create rejects an empty batch and one of more than 65535 fields (a grid
    dimension) before it reads any member (the dummy handles below are never dereferenced)."""
    n = 65536
    arr = (ctypes.c_void_p * n)(*([1] * n))
    h = ctypes.c_void_p()
    assert lib.sr_batch_create(arr, n, None, ctypes.byref(h)) == 1 and h.value is None
    assert b"65535" in lib.sr_last_error()
    assert lib.sr_batch_create(arr, 0, None, ctypes.byref(h)) == 1


def test_noise_weights_checks_arguments_before_device_use(lib):
    """sr_noise_weights validates pointers and sizes before any CUDA call (the dummy pointers
    below are never dereferenced)."""
    buf = (ctypes.c_float * 16)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    W = (ctypes.c_float * 8)()
    Wp = ctypes.cast(W, nat.P_float)
    call = lambda N, f, K, J, E, sg, s1, n, Wh, Wm: lib.sr_noise_weights(N, f, K, J, E, sg, s1, n, 0, Wh, Wm,
                                                                          None, None)
    assert call(16, 2, 5, 3, 1, None, p, 10, Wp, None) == 1          # no sigma
    assert call(16, 2, 5, 3, 1, p, p, 10, None, None) == 1           # no output
    assert call(16, 2, 5, 7, 1, p, p, 10, Wp, None) == 2             # 2 * 2^5 > F - 1
    assert call(16, 2, 5, 1, 1, p, p, 10, Wp, None) == 2             # J < 2
    assert call(16, 2, 5, 3, 1, p, p, 1, Wp, None) == 2              # one realisation
    assert call(0, 2, 5, 3, 1, p, p, 10, Wp, None) == 2
    assert call(16, 2, 0, 3, 1, p, p, 10, Wp, None) == 2
    assert call(16, 2, 5, 3, 0, p, p, 10, Wp, None) == 2
    assert b"sr_noise_weights" in lib.sr_last_error()


def test_struct_layouts_match_c(tmp_path):
    """ctypes mirrors of the header's structs have the C compiler's sizes and offsets."""
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "starred.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sr_problem_desc), offsetof(sr_problem_desc, lambda),
         offsetof(sr_problem_desc, conv_mode), sizeof(sr_layout), offsetof(sr_layout, total), sizeof(sr_optim_cfg),
         sizeof(sr_noise_timing), offsetof(sr_noise_timing, batch));
  printf("%zu %zu %zu %zu\\n", sizeof(sr_lbfgsb_cfg), offsetof(sr_lbfgsb_cfg, factr), sizeof(sr_lbfgsb_info),
         offsetof(sr_lbfgsb_info, pg_norm));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(nat.ProblemDesc), nat.ProblemDesc.lam.offset, nat.ProblemDesc.conv_mode.offset,
                    ctypes.sizeof(nat.Layout), nat.Layout.total.offset, ctypes.sizeof(nat.OptimCfg),
                    ctypes.sizeof(nat.NoiseTiming), nat.NoiseTiming.batch.offset,
                    ctypes.sizeof(nat.LbfgsbCfg), nat.LbfgsbCfg.factr.offset, ctypes.sizeof(nat.LbfgsbInfo),
                    nat.LbfgsbInfo.pg_norm.offset]
