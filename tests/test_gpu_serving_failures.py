"""Failure paths of the serving calls and of scene upload, through the C-ABI on a GB300.

Every failure here is made on the host: a context flag that makes each serving wave fail to
be issued (as if its wave state could not be allocated), a cancellation, an output larger than
the device, a scene with a NaN vertex.  No kernel is made to fault.
"""
import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S

pytestmark = pytest.mark.gpu

OOM, CANCELLED, INVALID, NOT_FOUND = -2, -9, -1, -6


@pytest.fixture(scope="module")
def hpt_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    return hpt


def test_failed_waves_reach_every_request(hpt_mod):
    hpt = hpt_mod
    ctx = hpt.Context(0, flags=hpt.CTX_FAIL_SERVING_WAVES)
    try:
        sid = ctx.upload_scene(S.config0_scene())
        rs = [S.config0_render(W=64, H=48, spp=4, K=2), S.config0_render(W=200, H=20, spp=8, K=1)]
        outs = [hpt.alloc_output(r) for r in rs]
        ids = [ctx.submit(sid, r, o) for r, o in zip(rs, outs)]
        for i in ids:
            with pytest.raises(hpt.HptError) as e:
                ctx.wait(i, 60000)
            assert e.value.status == OOM and "injected" in str(e.value)
            with pytest.raises(hpt.HptError) as e:
                ctx.poll(i)
            assert e.value.status == OOM
            t = ctx.request_times(i)
            assert t[0] <= t[1] <= t[2]
        ctx.sync()   # the device itself is fine
    finally:
        ctx.close()
    # a context without the flag serves the same requests
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config0_scene())
        r = S.config0_render(W=64, H=48, spp=4, K=2)
        ref = hpt.alloc_output(r)
        ctx.trace(sid, r, ref)
        ctx.sync()
        out = hpt.alloc_output(r)
        i = ctx.submit(sid, r, out)
        ctx.wait(i, 60000)
        assert ctx.poll(i)
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    finally:
        ctx.close()


def test_cancel_queued_and_running_requests(hpt_mod):
    hpt = hpt_mod
    ctx = hpt.Context(0, max_inflight=1)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        big = S.config1_render(W=1920, H=1080, spp=64, K=8)
        small = S.config1_render(W=96, H=64, spp=8, K=2)
        ref = hpt.alloc_output(small)
        ctx.trace(sid, small, ref)
        ctx.sync()
        o_big, o_q, o_ok = hpt.alloc_output(big), hpt.alloc_output(small), hpt.alloc_output(small)
        i_big = ctx.submit(sid, big, o_big)
        i_q = ctx.submit(sid, small, o_q)          # waits behind the running one (one slot)
        i_ok = ctx.submit(sid, small, o_ok)
        ctx.cancel(i_q)
        with pytest.raises(hpt.HptError) as e:
            ctx.wait(i_q, 1000)
        assert e.value.status == CANCELLED
        assert ctx.request_times(i_q)[1] == -1     # never admitted
        ctx.cancel(i_big)
        with pytest.raises(hpt.HptError) as e:
            ctx.wait(i_big, 120000)
        assert e.value.status == CANCELLED
        ctx.wait(i_ok, 120000)                     # the others still complete
        assert np.array_equal(o_ok.cpu().numpy(), ref.cpu().numpy())
        ctx.cancel(i_ok)                           # finished: left as it is
        assert ctx.poll(i_ok)
        with pytest.raises(hpt.HptError) as e:
            ctx.cancel(123456789)
        assert e.value.status == NOT_FOUND
        ctx.sync()
    finally:
        ctx.close()


def test_library_owned_outputs(hpt_mod):
    """out_dev == NULL: the output is allocated at admission, read back and released."""
    hpt = hpt_mod
    import torch
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        rs = [S.config1_render(W=203, H=117, spp=8, K=2), S.config1_render(W=64, H=40, spp=4, K=8)]
        refs = []
        for r in rs:
            o = hpt.alloc_output(r)
            ctx.trace(sid, r, o)
            ctx.sync()
            refs.append(o.cpu().numpy())
        ids = [ctx.submit(sid, r, None) for r in rs]
        for i, r, ref in zip(ids, rs, refs):
            ctx.wait(i, 120000)
            host = np.empty(r.out_shape(), np.complex64)
            ctx.request_output(i, host)
            assert np.array_equal(host, ref)
            dev = torch.empty(r.out_shape(), dtype=torch.complex64, device="cuda")
            ctx.request_output(i, dev)
            assert np.array_equal(dev.cpu().numpy(), ref)
            with pytest.raises(hpt.HptError) as e:
                ctx.request_output(i, np.empty(4, np.complex64))
            assert e.value.status == INVALID
            ctx.request_release(i)
            with pytest.raises(hpt.HptError) as e:
                ctx.poll(i)
            assert e.value.status == NOT_FOUND
        # an output larger than the device can ever hold is refused, not queued forever
        huge = S.config1_render(W=65536, H=32768, spp=1, K=8)
        i = ctx.submit(sid, huge, None)
        with pytest.raises(hpt.HptError) as e:
            ctx.wait(i, 60000)
        assert e.value.status == OOM
        ctx.sync()
    finally:
        ctx.close()


def test_scene_with_nan_vertex_is_rejected(hpt_mod):
    hpt = hpt_mod
    ctx = hpt.Context(0)
    try:
        for field in ("verts", "normals"):
            sc = S.config0_scene()
            a = getattr(sc, field).copy()
            a[2, 1] = np.nan
            setattr(sc, field, a)
            with pytest.raises(hpt.HptError) as e:
                ctx.upload_scene(sc)
            assert e.value.status == INVALID, field
        sc = S.config0_scene()
        sc.verts = sc.verts.copy()
        sc.verts[0, 0] = np.inf
        with pytest.raises(hpt.HptError) as e:
            ctx.upload_scene(sc)
        assert e.value.status == INVALID
        ctx.sync()
    finally:
        ctx.close()
