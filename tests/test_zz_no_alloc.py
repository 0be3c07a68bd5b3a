"""The fixed-scratch trace entry point (collected last on purpose).

hpt_trace_fixed_scratch serves callers that cannot allocate device memory while they run (a
real-time display loop that must not stall on cudaMalloc, or a process whose device memory is
handed out by another framework's pool): all of its scratch lives in one fixed device array
of the library, placed on the device when the context is created.  This test calls it through
the C-ABI and checks, twice in a row, that its fields equal those of hpt_trace bit for bit (the
array keeps the previous call's contents, so the second call shows that what must start at zero
is cleared) and that a call leaves the device's free memory unchanged.
"""
import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


def test_fixed_scratch_matches_trace_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        # ragged SLM, all materials, RGB, depth 4, K = 2: ~600k paths, more than one wave of
        # the fixed array
        r = S.config1_render(W=203, H=117, spp=8, K=2)
        outs = [hpt.alloc_output(r) for _ in range(2)]
        for prec in (hpt.PREC_DF32, hpt.PREC_FP64):
            ref = hpt.alloc_output(r)
            ctx.trace(sid, r, ref, precision=prec)
            ctx.sync()
            ref = ref.cpu().numpy()
            for call in range(2):
                out = outs[call]
                out.fill_(complex(float("nan"), float("nan")))
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
                ctx.trace_fixed_scratch(sid, r, out, precision=prec)
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free0, f"prec {prec} call {call}: device memory changed"
                ctx.sync()   # the kernels' status bits, including the fixed array's
                got = out.cpu().numpy()
                assert np.isfinite(got).all(), f"call {call}"
                assert np.array_equal(got, ref), f"fixed scratch prec={prec} call {call} differs from hpt_trace"
                assert_parity(got, ref, f"fixed scratch prec={prec} call {call}")
        # spp beyond the array's path capacity is rejected with a clear error
        big = S.config0_render(W=8, H=8, spp=1 << 22)
        with pytest.raises(hpt.HptError) as e:
            ctx.trace_fixed_scratch(ctx.upload_scene(S.config0_scene()), big, hpt.alloc_output(big))
        assert e.value.status == -1 and "fixed scratch" in str(e.value)
    finally:
        ctx.close()
