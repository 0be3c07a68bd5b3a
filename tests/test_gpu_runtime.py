"""Runtime forms of the trace on a GB300: captured frames (CUDA graphs) and the wave-size
autotuner must not change any field."""
import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _trace(ctx, sid, r, out, prec=1):
    ctx.trace(sid, r, out, precision=prec)
    ctx.sync()
    return out.cpu().numpy()


def test_graph_replay_equals_direct_launches(torch_cuda):
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    direct = hpt.Context(0, graphs=False)
    graphed = hpt.Context(0, graphs=True)
    try:
        sc = S.config1_scene()
        sd, sg = direct.upload_scene(sc), graphed.upload_scene(sc)
        r = S.config1_render(W=203, H=117, spp=8, K=4)
        od, og = hpt.alloc_output(r), hpt.alloc_output(r)
        for seed in (1, 2, 1):          # capture, replay with new job content, replay back
            r.seed = seed
            a = _trace(direct, sd, r, od)
            b = _trace(graphed, sg, r, og)
            assert np.array_equal(a, b), seed
        r2 = S.config1_render(W=203, H=117, spp=8, K=4, seed=2)
        assert not np.array_equal(_trace(direct, sd, r2, od), _trace(direct, sd, r, od))
    finally:
        direct.close()
        graphed.close()


def test_autotune_keeps_results(torch_cuda):
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=320, H=180, spp=8, K=2)
        out = hpt.alloc_output(r)
        before = _trace(ctx, sid, r, out)
        n = ctx.autotune(sid, S.config2_render())
        assert n in (1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 24)
        after = _trace(ctx, sid, r, out)
        assert np.array_equal(before, after)
    finally:
        ctx.close()
