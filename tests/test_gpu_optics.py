"""GB300 parity of the wave-optics steps against the FP64 oracle, through the C-ABI: the GRF phase
maps of Eq. 4, the angular spectrum propagation of the two-stage scheme, the trace in GRF phase
mode, and the two stages composed (trace to a recording plane, then ASM to the SLM)."""
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


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2606_14173_gb300 import build, hpt
    build.build()
    c = hpt.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def wo(oracle_mod):
    from oracle import waveoptics
    return waveoptics


def _wrapped(a, b):
    return np.abs(np.angle(np.exp(1j * (np.asarray(a, np.float64) - np.asarray(b, np.float64)))))


@pytest.mark.parametrize("nx,ny,K,off", [(512, 256, 3, 2), (64, 2048, 1, 0), (4096, 4096, 2, 5), (8192, 64, 1, 1),
                                           (2, 8, 2, 0)])
def test_grf_maps_match_the_oracle(ctx, wo, nx, ny, K, off):
    p = 6.4e-6
    phi = ctx.grf_build(7, K, nx, ny, p, hologram_offset=off)
    ctx.sync()
    got = phi.cpu().numpy()
    ref = wo.grf_maps(7, K, nx, ny, p, hologram_offset=off)
    d = _wrapped(got, ref)
    # arg r is ill-conditioned only where |r| ~ 0 (optical vortices): a 1e-6 fraction of points
    assert np.mean(d > 1e-3) <= 1e-4, np.mean(d > 1e-3)
    assert np.median(d) < 1e-5


def _field(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


@pytest.mark.parametrize("W,H,K,z", [(300, 200, 2, 12e-3), (37, 5, 1, -3e-3), (40, 24, 11, 5e-3),
                                       (4000, 6, 1, 2e-3), (1, 1, 2, 1e-3), (1920, 1080, 1, 80e-3)])
def test_asm_matches_the_oracle(ctx, wo, torch_cuda, W, H, K, z):
    torch = torch_cuda
    lams = (638e-9, 520e-9, 450e-9)
    rng = np.random.default_rng(W + H)
    U = _field(rng, (3, K, H, W))
    got = ctx.asm_propagate(torch.from_numpy(U).cuda(), lams, 6.4e-6, z)
    ctx.sync()
    ref = wo.asm_propagate(U, 6.4e-6, lams, z)
    assert_parity(got.cpu().numpy(), ref, f"asm {W}x{H} z={z}")


def test_asm_in_place(ctx, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(5)
    U = torch.from_numpy(_field(rng, (1, 3, 64, 96))).cuda()
    a = ctx.asm_propagate(U, (520e-9,), 8e-6, 5e-3)
    ctx.asm_propagate(U, (520e-9,), 8e-6, 5e-3, out=U)
    ctx.sync()
    assert torch.equal(a, U)


def test_trace_with_grf_phase(ctx, wo):
    """The cfg-1 scene with GRF phases (Eq. 4): GPU maps from hpt_grf_build in the GPU trace,
    the oracle's own maps in the oracle trace."""
    from oracle import Oracle
    from paper_2606_14173_gb300 import hpt
    sc = S.config1_scene()
    sid = ctx.upload_scene(sc)
    nx, ny = 4096, 2048
    for prec in (0, 1):
        r = S.config1_render(W=203, H=117, spp=8, K=4, hologram_offset=3, phase_mode=S.PHASE_GRF)
        r.grf = ctx.grf_build(r.phase_seed, r.K, nx, ny, r.pitch, hologram_offset=r.hologram_offset)
        out = hpt.alloc_output(r)
        ctx.trace(sid, r, out, precision=prec)
        ctx.sync()
        maps = wo.grf_maps(r.phase_seed, r.K, nx, ny, r.pitch, hologram_offset=r.hologram_offset)
        ref = Oracle(sc).trace_full(r, grf=maps)
        assert_parity(out.cpu().numpy(), ref, f"grf trace prec {prec}")
    ctx.release_scene(sid)


def test_two_stage_trace_then_asm(ctx, wo, torch_cuda):
    """Two-stage scheme (Sec. 5): the cfg-0 quads traced onto a recording plane 4 mm in front of
    the SLM (pose T moves the hologram plane to z = 4 mm), then propagated 4 mm to the SLM."""
    from oracle import Oracle
    from paper_2606_14173_gb300 import hpt
    sc = S.config0_scene()
    sid = ctx.upload_scene(sc)
    zw = 4e-3
    T = np.eye(4)
    T[2, 3] = -zw
    r = S.config0_render(W=160, H=120, spp=16, K=2, T=T)
    out = hpt.alloc_output(r)
    ctx.trace(sid, r, out, precision=0)
    slm = ctx.asm_propagate(out, r.lambdas, r.pitch, zw)
    ctx.sync()
    wrp = Oracle(sc).trace_full(r)
    ref = wo.asm_propagate(wrp, r.pitch, r.lambdas, zw)
    assert_parity(slm.cpu().numpy(), ref, "two-stage")
    ctx.release_scene(sid)


def test_invalid_arguments(ctx, torch_cuda):
    from paper_2606_14173_gb300 import hpt
    with pytest.raises(hpt.HptError):
        ctx.grf_build(1, 1, 300, 256, 6.4e-6)          # not a power of two
    with pytest.raises(hpt.HptError):
        ctx.grf_build(1, 1, 16384, 16, 6.4e-6)         # above 8192
    U = torch_cuda.zeros((1, 1, 8, 4097), dtype=torch_cuda.complex64, device="cuda")
    with pytest.raises(hpt.HptError):
        ctx.asm_propagate(U, (520e-9,), 8e-6, 1e-3)    # padded width above 8192
    U = torch_cuda.zeros((1, 1, 8, 8), dtype=torch_cuda.complex64, device="cuda")
    with pytest.raises(hpt.HptError):
        ctx.asm_propagate(U, (-1.0,), 8e-6, 1e-3)
    for lam, p, z in ((float("inf"), 8e-6, 1e-3), (520e-9, float("nan"), 1e-3), (520e-9, 8e-6, float("inf"))):
        with pytest.raises(hpt.HptError):
            ctx.asm_propagate(U, (lam,), p, z)
    with pytest.raises(hpt.HptError):
        ctx.grf_build(1, 1, 64, 64, float("inf"))
    ctx.sync()


@pytest.mark.parametrize("W,H,z", [(160, 120, 2e-3), (300, 37, -1e-3)])
def test_phase_encode_matches_the_oracle(ctx, wo, torch_cuda, W, H, z):
    """Gradient descent on the SLM phase under complex supervision: the GPU's iterates and
    losses follow the oracle's (the same start, target and step)."""
    torch = torch_cuda
    rng = np.random.default_rng(W)
    p, lam, iters = 8e-6, 520e-9, 12
    T = wo.asm_propagate(np.exp(1j * rng.uniform(-np.pi, np.pi, (H, W)))[None, None], p, [lam], z)[0, 0]
    T = T + 0.1 * (rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W)))
    phi0 = rng.uniform(-np.pi, np.pi, (H, W))
    lr = 0.1 / float(np.mean(np.abs(T) ** 2))
    Tg = torch.from_numpy(T.astype(np.complex64)).cuda()
    phi = torch.from_numpy(phi0.astype(np.float32)).cuda()
    L = ctx.phase_encode(Tg, phi, lam, p, z, iters, lr)
    ref_phi, ref_L = wo.encode(phi0.astype(np.float32).astype(np.float64), T.astype(np.complex64).astype(np.complex128),
                               p, lam, z, iters, lr)
    assert np.all(np.abs(L - ref_L) <= 1e-4 * ref_L), (L, ref_L)
    d = np.abs(np.angle(np.exp(1j * (phi.cpu().numpy() - ref_phi))))
    assert d.max() < 1e-3 and np.median(d) < 1e-5
    assert ref_L[-1] < ref_L[0]
