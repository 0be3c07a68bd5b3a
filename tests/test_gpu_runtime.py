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


def test_trace_into_host_memory_equals_device_trace(torch_cuda):
    """hpt_trace_host (the device trace into the context's staging buffer, then one copy to host
    memory) gives the device trace's fields bit for bit: for repeated calls (a captured frame
    replayed), with and without graphs, and after a larger request grows the staging buffer."""
    from paper_2606_14173_gb300 import hpt
    for graphs in (True, False):
        ctx = hpt.Context(0, graphs=graphs)
        try:
            sid = ctx.upload_scene(S.config1_scene())
            for W, H, K, seed in ((203, 117, 4, 1), (203, 117, 4, 2), (320, 180, 8, 3), (203, 117, 4, 1)):
                r = S.config1_render(W=W, H=H, spp=8, K=K, seed=seed)
                ref = _trace(ctx, sid, r, hpt.alloc_output(r))
                host = np.empty(ref.shape, np.complex64)
                ctx.trace_host(sid, r, host)
                assert np.array_equal(host, ref), (graphs, W, H, K, seed)
        finally:
            ctx.close()


def _ctx_with_wave_paths(n, **kw):
    import os
    from paper_2606_14173_gb300 import hpt
    old = os.environ.get("HPT_WAVE_PATHS")
    os.environ["HPT_WAVE_PATHS"] = str(n)
    try:
        return hpt.Context(0, **kw)
    finally:
        if old is None:
            del os.environ["HPT_WAVE_PATHS"]
        else:
            os.environ["HPT_WAVE_PATHS"] = old


def test_trace_into_pinned_host_memory_row_by_row(torch_cuda):
    """hpt_trace_host into pinned memory copies the rows each wave completes while later waves
    run.  Small waves whose item ranges end inside tiles and inside tile rows (spp 7 and 3), tile
    rows longer than a wave (a row finished only by the next wave), three wavelengths and sizes
    that are not multiples of the 8x4 tile: the host fields equal the device trace's bit for bit,
    every element written (the buffer starts as NaN), with and without captured graphs for the
    device trace, and after a larger request grows the staging buffer."""
    torch = torch_cuda
    from paper_2606_14173_gb300 import hpt
    sc = S.config1_scene()
    for paths, cases in ((65536, ((203, 117, 4, 7, 1), (320, 180, 8, 8, 2), (203, 117, 4, 7, 3))),
                         (4096, ((643, 21, 2, 3, 4), (203, 117, 1, 5, 5)))):
        for graphs in (True, False):
            ctx = _ctx_with_wave_paths(paths, graphs=graphs)
            try:
                sid = ctx.upload_scene(sc)
                for W, H, K, spp, seed in cases:
                    r = S.config1_render(W=W, H=H, spp=spp, K=K, seed=seed, max_depth=2)
                    ref = _trace(ctx, sid, r, hpt.alloc_output(r))
                    host = torch.empty(ref.shape, dtype=torch.complex64, pin_memory=True).numpy()
                    host[...] = np.nan
                    ctx.trace_host(sid, r, host)
                    assert np.array_equal(host, ref), (paths, graphs, W, H, K, spp, seed)
            finally:
                ctx.close()


def test_autotune_keeps_results(torch_cuda):
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=320, H=180, spp=8, K=2)
        out = hpt.alloc_output(r)
        before = _trace(ctx, sid, r, out)
        t = ctx.autotune(sid, S.config2_render())
        assert t["paths_per_wave"] in (1 << 21, 1 << 22, 1 << 23, 1 << 24)
        assert 1 <= t["lanes"] <= 4 and t["trace_blocks_per_sm"] >= 1 and t["shade_blocks_per_sm"] >= 1
        assert t["scene_class"] == 1 and t["candidates"] >= 4
        assert 0 < t["band_ms"] <= t["band_ms_start"] and t["band_path_samples"] >= 50_000_000
        after = _trace(ctx, sid, r, out)      # traced with the tuned shape of the scene's class
        assert np.array_equal(before, after)
        host = np.empty(after.shape, np.complex64)
        ctx.trace_host(sid, r, host)
        assert np.array_equal(host, before)
    finally:
        ctx.close()


def test_back_to_back_replays_keep_their_own_job_tables(torch_cuda):
    """Six replays of one captured frame queued without a host wait, each with another seed: each
    replay must read its own job table (the tables go through a ring of pinned buffers)."""
    from paper_2606_14173_gb300 import hpt
    torch = torch_cuda
    direct = hpt.Context(0, graphs=False)
    graphed = hpt.Context(0, graphs=True)
    try:
        sc = S.config1_scene()
        sd, sg = direct.upload_scene(sc), graphed.upload_scene(sc)
        r = S.config1_render(W=160, H=90, spp=4, K=2)
        out = hpt.alloc_output(r)
        stream = torch.cuda.current_stream()
        copies = []
        for seed in range(1, 7):
            r.seed = seed
            graphed.trace(sg, r, out, precision=1, stream=stream)
            copies.append(out.clone())          # same stream: ordered after this replay
        graphed.sync()
        torch.cuda.synchronize()
        od = hpt.alloc_output(r)
        for seed, c in zip(range(1, 7), copies):
            r.seed = seed
            assert np.array_equal(c.cpu().numpy(), _trace(direct, sd, r, od)), seed
    finally:
        direct.close()
        graphed.close()


def test_timed_trace_reports_kernels_and_keeps_results(torch_cuda):
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=320, H=180, spp=8, K=2)
        out = hpt.alloc_output(r)
        ref = _trace(ctx, sid, r, out)
        out.zero_()
        t = ctx.trace_timed(sid, r, out)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert set(t) == set(hpt.KERNEL_NAMES)
        waves = t["k_gen"][1]
        assert waves >= 1 and t["k_accum"][1] == waves
        # per iteration one coherent-ray and one incoherent/shadow-ray kernel of each kind
        assert t["k_trace"][1] == 2 * waves * (r.max_depth + 1)
        assert t["k_shade"][1] == t["k_trace"][1]
        assert all(ms > 0 for ms, _ in t.values())
    finally:
        ctx.close()


def test_counting_trace_meets_the_bar_against_the_trace(torch_cuda):
    """hpt_trace_counters runs separately compiled counting kernels: its fields need not be the
    trace's bit for bit, but they meet the parity bar against them, and its counts are those of
    the render (one path sample per (lambda, pixel, sample), at least one ray each)."""
    from paper_2606_14173_gb300 import hpt
    from tests.parity import assert_parity
    ctx = hpt.Context(0)
    try:
        sid = ctx.upload_scene(S.config1_scene())
        r = S.config1_render(W=320, H=180, spp=8, K=4)
        out = hpt.alloc_output(r)
        ref = _trace(ctx, sid, r, out)
        c = ctx.trace_counters(sid, r, out)
        assert_parity(out.cpu().numpy(), ref, "counting trace")
        assert c["samples"] == r.path_samples()
        assert c["rays"] >= c["samples"] and c["box_tests"] > c["rays"] and c["tri_tests"] > 0
        assert c["shadow_rays"] + c["bounces"] <= c["rays"]
    finally:
        ctx.close()


def test_many_waves_over_lanes_graph_and_direct(torch_cuda, oracle_mod):
    """A frame split into many small waves (65536 paths each) rotates over the wave lanes, in a
    captured graph and in direct launches: the two agree bit for bit and match the oracle."""
    import os
    from paper_2606_14173_gb300 import hpt
    from tests.parity import assert_parity
    old = os.environ.get("HPT_WAVE_PATHS")
    os.environ["HPT_WAVE_PATHS"] = "65536"
    try:
        direct = hpt.Context(0, graphs=False)
        graphed = hpt.Context(0, graphs=True)
    finally:
        if old is None:
            del os.environ["HPT_WAVE_PATHS"]
        else:
            os.environ["HPT_WAVE_PATHS"] = old
    try:
        sc = S.config1_scene()
        sd, sg = direct.upload_scene(sc), graphed.upload_scene(sc)
        r = S.config1_render(W=160, H=96, spp=8, K=2)        # 368640 paths: 6 waves
        od, og = hpt.alloc_output(r), hpt.alloc_output(r)
        a = _trace(direct, sd, r, od)
        for _ in range(2):                                    # capture, then replay
            b = _trace(graphed, sg, r, og)
            assert np.array_equal(a, b)
        assert_parity(a, oracle_mod.Oracle(sc).trace_full(r), "many waves")
    finally:
        direct.close()
        graphed.close()


def test_probe_peaks_are_plausible(torch_cuda):
    from paper_2606_14173_gb300 import hpt
    ctx = hpt.Context(0)
    try:
        p = ctx.probe_peaks()
        assert p["sms"] >= 1
        assert p["fp32_tflops"] > 1.0 and p["fp64_tflops"] > 0.01 and p["l2_read_gbs"] > 100.0
        assert p["fp64_tflops"] < p["fp32_tflops"]
    finally:
        ctx.close()
