"""GB300 ambient-cache construction (texture baking) through the C-ABI against the FP64 oracle:
the furnace closed form, the cfg-1 scene cell by cell, and a cache set on the device and read
by the trace (the "fast" variant)."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu
MM = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    c = hpt.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("depth", [1, 2, 4])
def test_bake_furnace(ctx, depth):
    rho, Le = 0.5, 1.0
    sid = ctx.upload_scene(S.furnace_scene(albedo=rho, Le=Le))
    E = ctx.cache_bake(sid, 6, [-3 * MM, -3 * MM, -1 * MM], [3 * MM, 3 * MM, 5 * MM], 16, depth, seed=4)
    ctx.sync()
    want = math.pi * Le * (1 - rho ** depth) / (1 - rho)
    got = E.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 2e-6 * want
    ctx.release_scene(sid)


def test_bake_matches_the_oracle(ctx, oracle_mod):
    """The cfg-1 scene (mirrors, glass, GGX, Lambert under one area light), 16^3 cells x RGB x
    32 directions, depth 3: the same Philox draws on both sides, the GPU in float32 from the
    cell centre on (a bake path has no coherent part).  The bar is the trace's, with the same
    exception: a cell-channel beyond 1e-4 is excused only when the oracle finds it float32-
    sensitive -- moving the cell centre within the 32-ulp float32 budget of a path changes it
    by at least the tolerance -- and the disagreement stays within tolerance + that bound;
    unexplained cell-channels <= 0.1 %."""
    sc = S.config1_scene()
    sid = ctx.upload_scene(sc)
    lo, hi = [-10 * MM, -3 * MM, 3 * MM], [10 * MM, 8 * MM, 32 * MM]
    res, spp, depth = 16, 32, 3
    E = ctx.cache_bake(sid, res, lo, hi, spp, depth, seed=11)
    ctx.sync()
    got = E.cpu().numpy().reshape(-1, 3).astype(np.float64)
    lo32, hi32 = np.float32(lo).astype(np.float64), np.float32(hi).astype(np.float64)
    orc = oracle_mod.Oracle(sc)
    ref = orc.bake(res, lo32, hi32, spp, depth, seed=11)
    scale = max(float(np.abs(ref).mean()), 1e-30)
    tol = 1e-4 * np.maximum(np.abs(ref), 1e-3 * scale)
    bad = np.abs(got - ref) > tol
    cells = np.nonzero(bad.any(axis=1))[0]
    _, sens = orc.bake(res, lo32, hi32, spp, depth, seed=11, cells=cells, with_sens=True)
    sv = np.zeros_like(ref)
    sv[cells] = sens
    explained = bad & (sv >= tol) & (np.abs(got - ref) <= tol + sv)
    unexplained = int((bad & ~explained).sum())
    print(f"bake: {int(bad.sum())} of {bad.size} cell-channels beyond 1e-4, {unexplained} unexplained")
    assert unexplained <= 1e-3 * bad.size, (int(bad.sum()), unexplained)
    assert abs(got.mean() - ref.mean()) <= 5e-4 * abs(ref.mean())
    ctx.release_scene(sid)


def test_set_cache_then_trace(ctx, oracle_mod, torch_cuda):
    """A seeded float grid set as the cache on the device (rounded to binary16 there) and the
    same grid rounded by numpy in the oracle's scene: the traced fields with the cache agree."""
    torch = torch_cuda
    from paper_2606_14173_gb300 import hpt
    base = S.config1_scene()
    sid = ctx.upload_scene(base)
    res = 32
    lo, hi = np.float32([-20 * MM, -3 * MM, 0.0]), np.float32([20 * MM, 15 * MM, 40 * MM])
    grid = (np.random.default_rng(8).uniform(0.5, 3.0, (res, res, res, 3))).astype(np.float32)
    ctx.set_cache(sid, torch.from_numpy(grid).cuda(), lo, hi)
    r = S.config1_render(W=128, H=96, spp=8, K=2, use_cache=1)
    out = hpt.alloc_output(r)
    ctx.trace(sid, r, out, precision=1)
    ctx.sync()
    sc = dataclasses.replace(base, cache_res=res, cache_bmin=lo, cache_bmax=hi, cache_E=grid.astype(np.float16))
    ref = oracle_mod.Oracle(sc).trace_full(r)
    assert_parity(out.cpu().numpy(), ref, "set_cache trace")
    ctx.set_cache(sid, None, lo, hi)
    with pytest.raises(hpt.HptError):
        ctx.trace(sid, r, out, precision=1)
    ctx.sync()
    ctx.release_scene(sid)


def test_fast_variant_pipeline(ctx, torch_cuda):
    """Bake the cache on the GPU, set it, trace with it: every field finite, and the cache
    changes the result."""
    from paper_2606_14173_gb300 import hpt
    sid = ctx.upload_scene(S.config1_scene())
    lo, hi = [-20 * MM, -3 * MM, 0.0], [20 * MM, 15 * MM, 40 * MM]
    E = ctx.cache_bake(sid, 24, lo, hi, 16, 3, seed=2)
    ctx.set_cache(sid, E, lo, hi)
    r0 = S.config1_render(W=96, H=64, spp=8, K=1, use_cache=0)
    r1 = S.config1_render(W=96, H=64, spp=8, K=1, use_cache=1)
    a, b = hpt.alloc_output(r0), hpt.alloc_output(r1)
    ctx.trace(sid, r0, a)
    ctx.trace(sid, r1, b)
    ctx.sync()
    A, B = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(np.isfinite(B)) and not np.array_equal(A, B)
    ctx.release_scene(sid)


def test_bake_invalid_arguments(ctx, torch_cuda):
    from paper_2606_14173_gb300 import hpt
    sid = ctx.upload_scene(S.config0_scene())
    with pytest.raises(hpt.HptError):
        ctx.cache_bake(sid, 0, [0, 0, 0], [1, 1, 1], 4, 2)
    with pytest.raises(hpt.HptError):
        ctx.cache_bake(sid, 4, [0, 0, 0], [1, 0, 1], 4, 2)
    with pytest.raises(hpt.HptError):
        ctx.cache_bake(sid + 1000, 4, [0, 0, 0], [1, 1, 1], 4, 2)
    ctx.sync()
    ctx.release_scene(sid)


def test_cache_upload_from_host_equals_device_set(ctx, torch_cuda):
    """The same binary16 grid uploaded from host memory and set from a device float grid (whose
    values are exactly representable in binary16) gives the same traced fields bit for bit."""
    torch = torch_cuda
    from paper_2606_14173_gb300 import hpt
    base = S.config1_scene()
    a_sid, b_sid = ctx.upload_scene(base), ctx.upload_scene(base)
    res = 16
    lo, hi = [-20 * MM, -3 * MM, 0.0], [20 * MM, 15 * MM, 40 * MM]
    grid16 = np.random.default_rng(9).uniform(0.5, 3.0, (res, res, res, 3)).astype(np.float16)
    ctx.cache_upload(a_sid, grid16, lo, hi)
    ctx.set_cache(b_sid, torch.from_numpy(grid16.astype(np.float32)).cuda(), lo, hi)
    r = S.config1_render(W=96, H=64, spp=8, K=1, use_cache=1)
    oa, ob = hpt.alloc_output(r), hpt.alloc_output(r)
    ctx.trace(a_sid, r, oa)
    ctx.trace(b_sid, r, ob)
    ctx.sync()
    assert torch.equal(oa, ob)
    ctx.release_scene(a_sid)
    ctx.release_scene(b_sid)
