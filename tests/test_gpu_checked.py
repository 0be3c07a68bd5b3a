"""The checked build of the library on a GB300.

The same sources built with -DHPT_CHECKED=1: every device index into the path state, the queues,
the BVH and the triangle arrays is checked before use, and a failing check sets a status bit
(reported by hpt_sync as HPT_ERR_DEVICE, "index-out-of-bounds") and skips the access instead of
faulting.  Traces of the 30-sphere scene, the 185k-triangle cache scene and a scene whose every
coherent ray takes the double-precision fallback, in both arithmetics, must leave no bit set, and
their fields must meet the parity bar against the product build's.  The checked library runs in a
child process (HPT_LIB), so that this process keeps the product library.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, sys.argv[2])
import numpy as np
from paper_2606_14173_gb300 import hpt
from tests.test_gpu_checked import cases
assert hpt.LIB_PATH.endswith("libhpt_checked.so"), hpt.LIB_PATH
ctx = hpt.Context(0)
out = {}
for name, sc, r in cases():
    sid = ctx.upload_scene(sc)
    o = hpt.alloc_output(r)
    for prec in (0, 1):
        ctx.trace(sid, r, o, precision=prec)
        ctx.sync()                      # raises on any status bit
        out[f"{name}_{prec}"] = o.cpu().numpy()
ctx.close()
np.savez(sys.argv[1], **out)
"""


def cases():
    from tests.test_gpu_fallback import _stack_scene
    return [("cfg1", S.config1_scene(), S.config1_render(W=203, H=117, spp=8, K=2)),
            ("cfg3", S.config3_scene(), S.config3_render(W=96, H=64, spp=4, K=2)),
            ("stack", _stack_scene(), S.config0_render(W=96, H=96, spp=8, K=1))]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_checked_build_sets_no_bounds_bit_and_meets_the_bar(torch_cuda, tmp_path):
    from paper_2606_14173_gb300 import build, hpt
    lib = build.build(checked=True)
    res = tmp_path / "checked.npz"
    env = dict(os.environ, HPT_LIB=lib)
    p = subprocess.run([sys.executable, "-c", CHILD, str(res), ROOT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    got = np.load(res)
    ctx = hpt.Context(0)
    try:
        for name, sc, r in cases():
            sid = ctx.upload_scene(sc)
            o = hpt.alloc_output(r)
            for prec in (0, 1):
                ctx.trace(sid, r, o, precision=prec)
                ctx.sync()
                assert_parity(got[f"{name}_{prec}"], o.cpu().numpy(), f"checked build {name} prec {prec}")
    finally:
        ctx.close()
