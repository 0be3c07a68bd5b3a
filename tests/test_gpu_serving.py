"""Serving (continuous batching) through the C-ABI on a GB300.

Requests of different scenes, SLM sizes, sample counts, hologram counts, arithmetics and
poses are submitted together; the scheduler batches their work items into shared waves.
Each request's fields must equal those of the same request traced alone (the per-pixel
estimate does not depend on how items are batched), within the parity tolerance -- in fact
bitwise.
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


def _pose(dx, dy):
    T = np.eye(4)
    T[0, 3], T[1, 3] = -dx, -dy
    return T


def _mix():
    return [
        ("cfg0", S.config0_render(W=256, H=256, spp=16, K=1), 1),
        ("cfg1", S.config1_render(W=203, H=117, spp=8, K=4), 1),
        ("cfg1", S.config1_render(W=512, H=512, spp=4, K=8, T=_pose(2e-3, -1e-3)), 0),
        ("cfg0", S.config0_render(W=96, H=64, spp=32, K=8, phase_mode=S.PHASE_ZERO), 0),
        ("cfg1", S.config1_render(W=64, H=48, spp=16, K=1, lambdas=(520e-9,), channels=(1,)), 1),
        ("cfg0", S.config0_render(W=300, H=20, spp=3, K=2, hologram_offset=5), 1),
    ]


def test_results_alone_and_in_the_mix(torch_cuda):
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    ctx = hpt.Context(0)
    try:
        sids = {"cfg0": ctx.upload_scene(S.config0_scene()), "cfg1": ctx.upload_scene(S.config1_scene())}
        mix = _mix()
        alone = []
        for name, r, prec in mix:
            out = hpt.alloc_output(r)
            ctx.trace(sids[name], r, out, precision=prec)
            ctx.sync()
            alone.append(out.cpu().numpy())
        outs = [hpt.alloc_output(r) for _, r, _ in mix]
        for o in outs:
            o.fill_(complex(float("nan"), float("nan")))
        torch_cuda.cuda.synchronize()
        ids = [ctx.submit(sids[name], r, o, precision=prec) for (name, r, prec), o in zip(mix, outs)]
        for i in ids:
            ctx.wait(i, 120000)
            assert ctx.poll(i)
        for (name, r, prec), i, o, ref in zip(mix, ids, outs, alone):
            got = o.cpu().numpy()
            assert_parity(got, ref, f"served {name} {r.W}x{r.H}")
            assert np.array_equal(got, ref), "batching changed the bits of a request"
            t = ctx.request_times(i)
            assert 0 <= t[0] <= t[1] <= t[2]
        ctx.sync()
    finally:
        ctx.close()


def test_config4_requests_alone_and_in_the_mix(torch_cuda):
    """Requests drawn by the config-4 recipe (each config's scene, pitch, wavelengths and depth, the
    185k-triangle scene with its ambient cache resident, poses and focal depths), shrunk to small
    SLMs and sample counts: library-owned outputs, each bit-identical to the same render traced
    alone."""
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        sids = {"cfg0": ctx.upload_scene(S.config0_scene()), "cfg1": ctx.upload_scene(S.config1_scene()),
                "cfg3": ctx.upload_scene(S.config3_scene())}
        reqs = []
        for key, r in S.config4_requests(40, seed=77):
            r.W, r.H, r.spp = max(8, r.W // 16), max(8, r.H // 16), max(2, r.spp // 16)
            reqs.append((key, r))
            if len(reqs) == 8:
                break
        assert {k for k, _ in reqs} >= {"cfg1", "cfg3"}
        alone = []
        for key, r in reqs:
            out = hpt.alloc_output(r)
            ctx.trace(sids[key], r, out)
            ctx.sync()
            alone.append(out.cpu().numpy())
        ids = [ctx.submit(sids[key], r, None) for key, r in reqs]
        for i, (key, r), ref in zip(ids, reqs, alone):
            ctx.wait(i, 120000)
            got = np.empty(r.out_shape(), np.complex64)
            ctx.request_output(i, got)
            ctx.request_release(i)
            assert np.array_equal(got, ref), f"{key} {r.W}x{r.H} spp {r.spp} K {r.K} differs in the mix"
        ctx.sync()
    finally:
        ctx.close()


def test_admission_by_memory_budget(torch_cuda):
    """With a budget smaller than two outputs, requests run one after another."""
    from paper_2606_14173_gb300 import hpt
    r = S.config0_render(W=256, H=256, spp=32, K=8)
    ctx = hpt.Context(0, hbm_budget_bytes=hpt.out_bytes(r) + 1, max_inflight=4)
    try:
        sid = ctx.upload_scene(S.config0_scene())
        outs = [hpt.alloc_output(r) for _ in range(3)]
        ids = [ctx.submit(sid, r, o) for o in outs]
        for i in ids:
            ctx.wait(i, 120000)
        times = [ctx.request_times(i) for i in ids]
        for a, b in zip(times, times[1:]):
            assert b[1] >= a[2] - 1e-6, (a, b)      # admitted only after the previous one finished
        ref = outs[0].cpu().numpy()
        for o in outs[1:]:
            assert np.array_equal(o.cpu().numpy(), ref)
    finally:
        ctx.close()


def test_wait_timeout_and_unknown_ids(torch_cuda):
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=960, H=540, spp=64, K=8)
        out = hpt.alloc_output(r)
        i = ctx.submit(sid, r, out)
        with pytest.raises(hpt.HptError) as e:
            ctx.wait(i, 1)
        assert e.value.status in (-4,)          # still running after 1 ms
        ctx.wait(i, 120000)
        with pytest.raises(hpt.HptError) as e:
            ctx.poll(987654)
        assert e.value.status == -6
        with pytest.raises(hpt.HptError) as e:
            ctx.release_scene(sid + 99)
        assert e.value.status == -6
    finally:
        ctx.close()


def test_bounded_queue_answers_busy(torch_cuda):
    """With one request on the device and room for one waiting, a burst of four submissions
    gets HPT_ERR_BUSY for at least one (nothing is queued for it); the accepted ones complete
    with the fields of the same request traced alone, and the queue takes requests again once
    it has drained."""
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0, max_inflight=1, max_queue=1)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=960, H=540, spp=64, K=8)
        ref = hpt.alloc_output(r)
        ctx.trace(sid, r, ref)
        ctx.sync()
        outs = [hpt.alloc_output(r) for _ in range(4)]
        ids, busy = [], 0
        for o in outs:
            try:
                ids.append((ctx.submit(sid, r, o), o))
            except hpt.HptError as e:
                assert e.status == -5, e
                busy += 1
        assert busy >= 1 and len(ids) >= 1
        for i, o in ids:
            ctx.wait(i, 120000)
            assert torch_cuda.equal(o, ref)
        i = ctx.submit(sid, r, outs[0])
        ctx.wait(i, 120000)
        assert torch_cuda.equal(outs[0], ref)
    finally:
        ctx.close()
