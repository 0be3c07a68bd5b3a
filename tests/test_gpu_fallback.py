"""The double-precision fallback traversal on a GB300 against the FP64 oracle.

Six coincident emissive triangles of different emission (a stack: every ray that meets it meets
all six at the same distance) in front of an emissive textured background.  The float traversal
of a coherent ray records tied hits as candidates; six overflow the candidate list, so every ray
through the stack is decided by the full traversal with exact triangle tests (and float tests of
widened boxes), whose tie rule -- the lowest triangle id -- picks the emission the oracle picks.
The counters show that the fallback ran; the fields must pass the parity bar in both coherent
arithmetics.
"""
import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _stack_scene():
    rng = np.random.default_rng(2024)
    b = S._Builder("coincident-stack")
    t = b.texture(rng.uniform(0.2, 1.0, (32, 32, 3)))
    back = b.material(S.LAMBERT, albedo=(1.0, 1.0, 1.0), Le=(1.0, 1.0, 1.0), tex=t, emit_tex=1)
    b.quad(np.array([-1.5, -1.5, 10.0]) * S.MM, np.array([3.0, 0, 0]) * S.MM, np.array([0, 3.0, 0]) * S.MM, back,
           flip=True)
    # a triangle over half of the view, facing the SLM (-z), six times with distinct emission
    v = np.array([[-1.2, -1.2, 5.0], [1.2, -1.2, 5.0], [-1.2, 1.2, 5.0]]) * S.MM
    for k in range(6):
        m = b.material(S.LAMBERT, albedo=(1.0, 1.0, 1.0), Le=(1.0 + k, 2.0 + 0.5 * k, 3.0 - 0.4 * k))
        b.mesh(v.copy(), np.tile([0.0, 0.0, -1.0], (3, 1)), np.zeros((3, 2)), [[0, 2, 1]], m)
    return b.build()


def test_fallback_traversal_matches_the_oracle(torch_cuda, oracle_mod):
    from paper_2606_14173_gb300 import hpt
    sc = _stack_scene()
    r = S.config0_render(W=192, H=192, spp=32, K=2)
    ref = oracle_mod.Oracle(sc).trace_full(r)
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(sc)
        out = hpt.alloc_output(r)
        c = ctx.trace_counters(sid, r, out)
        # the rays through the stack: about half of the 192 x 192 x 32 primary rays
        assert c["fp64_fallbacks"] > 100000 and c["refines"] >= c["fp64_fallbacks"]
        for prec in (0, 1):
            ctx.trace(sid, r, out, precision=prec)
            ctx.sync()
            assert_parity(out.cpu().numpy(), ref, f"stack prec {prec}")
    finally:
        ctx.close()
