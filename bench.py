"""Benchmark of the wave path tracer on the headline workload.

Workload: the 30-icosphere scene (~24k triangles, Lambertian / GGX / mirror / dielectric, one
area light), 1920x1080 SLM at 6.4 um, RGB (638/520/450 nm), 64 spp, depth 4, K = 8
Path-Reuse holograms: 398 M path samples per step.  One step = one full hologram set.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = path samples / s over the whole job (all ranks); the plain
form (FP64 coherent arithmetic, one launch per wavelength) is timed beside the mixed-precision
batched form (double-float coherent arithmetic, all wavelengths and holograms in one launch).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "path samples/s & 1080p RGB K=8 holograms/s vs plain FP64 form; p50/p99 latency"
UNIT = "path samples/s"
# FP32 ALU peak of a GB300 from its unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop/FMA
# x 2.07 GHz (maximum SM clock).
SM_COUNT, FP32_LANES, SM_MHZ_MAX = 152, 128, 2070.0
def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


HBM_PEAK_GBS = _hbm_peak()
ALU_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12
# algorithmic FP32 work per counted event: 20 flop per child-box slab test (two per node visit),
# 30 per float ray-triangle test, 400 per coherent re-decision in double-float, 120 per
# incoherent vertex (shadow ray or BSDF bounce), 25 per hologram of a path sample (phase + Kahan sum)
FLOP_PER = {"box_tests": 20, "tri_tests": 30, "refines": 400, "vertex": 120, "hologram": 25}
# DRAM bytes (read + write) per k_trace launch: the average over every launch of both trace
# kernels in one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the 1920x270 band
# of the 30-sphere scene with 2,097,152-path waves (the first 120 launches), scaled by 4.0 to the
# 8,388,608-path waves of the headline frame (the traffic is per ray), copied here: the bench
# cannot read hardware counters itself.  None whenever k_trace changed since that capture.
TRACE_DRAM_BYTES_PER_LAUNCH = 138e6
# Issue counters of the two trace kernels from one ncu --set full capture each on the same band
# (coherent rays at iteration 0, incoherent and shadow rays at iteration 1), copied here for the
# same reason: threads active per issued warp instruction (smsp__thread_inst_executed_per_inst_
# executed / 32) and issue activity (smsp__issue_active).  None whenever k_trace changed since.
TRACE_ISSUE = {"simt_efficiency": {"coherent": 12.24 / 32, "incoherent_shadow": 13.44 / 32},
               "issue_active": {"coherent": 0.619, "incoherent_shadow": 0.662}}


# name -> (description, scene factory, render factory)
WORKLOADS = {
    "cfg2": ("cfg2: 30-icosphere scene (~24k tris, Lambert/GGX/mirror/dielectric, 1 area light), 1920x1080 SLM 6.4 um, "
             "RGB 638/520/450 nm, 64 spp, depth 4, K=8", "config1_scene", ("config2_render", {})),
    "band": ("profiling case: the cfg2 scene and SLM pitch, a 1920x270 band at mid height, RGB, 16 spp, depth 4, K=8",
             "config1_scene", ("config2_render", {"H": 270, "spp": 16})),
    "cfg3": ("cfg3: ~185k tris (icospheres + subdivided GGX/dielectric slabs), 128^3 binary16 ambient cache past the "
             "first bounce, 3840x2160 SLM 3.74 um, RGB, 256 spp, depth 4, K=8", "config3_scene", ("config3_render", {})),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-counters", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--cfg4-requests", type=int, default=2000, help="requests of the config-4 serving stream")
    p.add_argument("--serving-sweep", default="",
                   help="comma-separated offered rates (req/s): run only the config-4 bounded-admission sweep")
    p.add_argument("--sweep-requests", type=int, default=200)
    p.add_argument("--no-optics", action="store_true")
    p.add_argument("--workload", default="cfg2", choices=list(WORKLOADS),
                   help="cfg2 = the headline workload; the others are smaller cases of the same kernels for profiling")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def wait_ready(self, timeout=20.0):
        """Block until the first sample arrived: nvidia-smi's start-up (NVML initialisation) can
        hold the GPU for a fraction of a second, which must not fall into a timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.rows and time.perf_counter() - t0 < timeout:
            time.sleep(0.05)

    def window(self, t_begin, t_end):
        """Keep the samples taken between t_begin and t_end (perf_counter seconds) only: the
        sampler starts before the warm-up so that its own start-up overlaps no timed step."""
        self.t_window = (t_begin, t_end)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        tw = getattr(self, "t_window", None)
        for t, r in self.rows:
            if tw is not None and not (tw[0] - 0.2 <= t <= tw[1] + 0.2):
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    """Max over ranks (the timing rule: the slowest replica sets the whole job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Replicas only: every rank renders its own frame of the same workload with its own
    sampling seed; there is no exchange between ranks on the data path."""
    return 1 + rank


def job_value(samples_per_step, steps, max_ms, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * samples_per_step * steps / (max_ms / 1e3)


def cpu_oracle_rate(scene, r, n_pixels, seed=5):
    """The FP64 oracle as it stands, on all host cores, over a seeded pixel sample."""
    import oracle
    o = oracle.Oracle(scene)
    rng = np.random.default_rng(seed)
    pix = rng.choice(r.W * r.H, n_pixels, replace=False)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    U = o.trace(r, pix, n_threads=cores)
    dt = time.perf_counter() - t0
    samples = n_pixels * len(r.lambdas) * r.spp
    return samples / dt, dt, cores, samples, pix, U


def precision_report(U, ref, flags_of=None):
    """Error of GPU fields U[lambda][m][pixel] against the FP64 oracle's ref, per output: the
    fraction of pixels within 1e-4 relative error and 1e-3 rad (where |ref| < 1e-3 RMS the bound
    is 1e-4 RMS; the phase is checked where |ref| >= 0.1 RMS), the median and maximum relative
    error and the maximum phase error.  flags_of(pixel indices) -> (flags, sens) of the oracle
    for those pixels: the pixels out of the bar are then counted by what the oracle flags in
    them (an edge or tie hit, an ill-conditioned incoherent part, an incoherent path through a
    mirror or dielectric, or a field that float32-sized moves of the image points change by the
    tolerance), and the ones it does not flag are counted as unattributed."""
    out, fails = [], []
    for l in range(U.shape[0]):
        for m in range(U.shape[1]):
            u, q = np.asarray(U[l, m], np.complex128), np.asarray(ref[l, m], np.complex128)
            rms = float(np.sqrt(np.mean(np.abs(q) ** 2)))
            a, d = np.abs(q), np.abs(u - q)
            rel = np.where(a < 1e-3 * rms, d / max(rms, 1e-300), d / np.maximum(a, 1e-300))
            ph = np.where(a >= 0.1 * rms, np.abs(np.angle(u * np.conj(q))), 0.0)
            ok = (rel <= 1e-4) & (ph <= 1e-3)
            out.append({"lambda": l, "m": m, "pass_frac": float(ok.mean()), "median_rel": float(np.median(rel)),
                        "max_rel": float(rel.max()), "max_phase_rad": float(ph.max())})
            tol = 1e-4 * np.maximum(a, 1e-3 * rms)
            fails += [(l, int(i), float(tol[i])) for i in np.nonzero(~ok)[0]]
    rep = {"outputs": out, "min_pass_frac": min(x["pass_frac"] for x in out),
           "max_phase_rad": max(x["max_phase_rad"] for x in out), "pixels": int(U.shape[2]),
           "failing_pixel_outputs": len(fails)}
    if flags_of is not None and fails:
        pix = sorted({i for _, i, _ in fails})
        fl, sens = flags_of(np.asarray(pix))
        col = {p: k for k, p in enumerate(pix)}
        cats = {"near_edge": 0, "ill_conditioned": 0, "incoherent_delta": 0, "sensitive_only": 0, "unattributed": 0}
        for l, i, tol in fails:
            f, sv = int(fl[l, col[i]]), float(sens[l, col[i]])
            if f & 0xFFFF: cats["near_edge"] += 1
            elif (f >> 16) & 0xFFFF: cats["ill_conditioned"] += 1
            elif (f >> 32) & 0xFFFF: cats["incoherent_delta"] += 1
            elif sv >= tol: cats["sensitive_only"] += 1
            else: cats["unattributed"] += 1
        rep["failing_by_oracle_flag"] = cats
    return rep


def run_optics(ctx, hpt, torch, r, out, sid, stream, reps=3):
    """The wave-optics steps around the tracer on the headline output: the K GRF phase maps of
    Eq. 4 (4096 x 2048 grid of the SLM pitch), the angular-spectrum propagation of all
    n_lambda x K fields over 80 mm (the two-stage scheme; 4096 x 4096 padded), and a traced
    frame in GRF phase mode.  Device time from CUDA events on the bench stream."""
    def timed_ms(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    nx, ny = 4096, 2048
    grf = {}
    grf_ms = timed_ms(lambda: grf.__setitem__("phi", ctx.grf_build(r.phase_seed, r.K, nx, ny, r.pitch, stream=stream)))
    res = torch.empty_like(out)
    asm_ms = timed_ms(lambda: ctx.asm_propagate(out, r.lambdas, r.pitch, 80e-3, out=res, stream=stream))
    Wp = Hp = 4096
    n_fields = len(r.lambdas) * r.K
    # algorithmic bytes of the row-column ASM that skips the zero padding: every field read and
    # written once; its spectrum (H rows of Wp) written by the forward x pass, read and written
    # by the y pass (FFT, transfer, inverse FFT, the window's rows kept) and read by the inverse
    # x pass; the transfer function of each wavelength read once
    alg = n_fields * 8 * (2 * r.W * r.H + 4 * Wp * r.H) + len(r.lambdas) * 8 * Wp * Hp
    achieved = alg / (asm_ms / 1e3) / 1e9
    rg = dataclasses.replace(r, phase_mode=2, grf=grf["phi"])
    grf_trace_ms = timed_ms(lambda: ctx.trace(sid, rg, out, precision=hpt.PREC_DF32, stream=stream))
    # ambient cache construction over the scene box: 128^3 cells x RGB x 16 directions, depth 3
    res, bspp, bdepth = 128, 16, 3
    lo, hi = [-20e-3, -3e-3, 0.0], [20e-3, 15e-3, 40e-3]
    bake = {}
    bake_ms = timed_ms(lambda: bake.__setitem__("E", ctx.cache_bake(sid, res, lo, hi, bspp, bdepth, seed=5,
                                                                      stream=stream)))
    bake_paths = res ** 3 * 3 * bspp
    # phase-only encoding of the green hologram (m = 0) under complex supervision, 10 steps
    tgt = out[1, 0].contiguous()
    phi = torch.zeros((r.H, r.W), dtype=torch.float32, device=out.device)
    enc_iters = 10
    enc_ms = timed_ms(lambda: ctx.phase_encode(tgt, phi, r.lambdas[1], r.pitch, 0.0, enc_iters,
                                               0.1 / float(torch.mean(tgt.abs() ** 2)), stream=stream))
    return {
        "phase_encode": {"field": [r.W, r.H], "iters": enc_iters, "ms": enc_ms, "ms_per_iter": enc_ms / enc_iters},
        "cache_bake": {"cells": res ** 3, "channels": 3, "directions": bspp, "max_depth": bdepth, "ms": bake_ms,
                       "paths_per_s": bake_paths / (bake_ms / 1e3)},
        "grf_maps": {"K": r.K, "grid": [nx, ny], "ms": grf_ms, "maps_per_s": r.K / (grf_ms / 1e3)},
        "asm": {"fields": n_fields, "field": [r.W, r.H], "padded": [Wp, Hp], "z_m": 80e-3, "ms": asm_ms,
                "fields_per_s": n_fields / (asm_ms / 1e3),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                             "frac": achieved / HBM_PEAK_GBS, "traffic": None,
                             "alg_bytes_per_field": alg / n_fields,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"}},
        "grf_phase_trace": {"ms_per_frame": grf_trace_ms,
                            "path_samples_per_s": r.path_samples() / (grf_trace_ms / 1e3)},
        "workload": "headline output (1920x1080, RGB, K = 8): GRF maps 4096x2048, ASM of 24 fields over 80 mm, "
                    "one frame traced with GRF phases; 128^3 ambient cache baked over the 30-sphere scene; "
                    "10 phase-only encoding steps of one 1080p hologram (z = 0, 4096^2 padded ASM both ways)",
    }


def serve_owned(ctx, hpt, requests, rate, seed):
    """Submit requests with Poisson arrivals at 'rate' per second, outputs owned by the library
    (allocated at admission by free HBM), and release each as it finishes.  requests: list of
    (scene id, render).  Returns latency and throughput statistics of the completed requests."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(requests))
    ctx.sync()
    outstanding, done, rejected = {}, [], 0

    def reap(block):
        for i in list(outstanding):
            if block:
                ctx.wait(i, 600000)
            elif not ctx.poll(i):
                continue
            done.append((ctx.request_times(i), outstanding.pop(i)))
            ctx.request_release(i)

    t_next = time.perf_counter()
    for (sid, r), g in zip(requests, gaps):
        t_next += g
        while True:
            dt = t_next - time.perf_counter()
            if dt <= 0:
                break
            reap(False)
            time.sleep(min(dt, 0.004))
        try:
            outstanding[ctx.submit(sid, r, None, precision=hpt.PREC_DF32)] = r
        except hpt.HptError as e:
            if e.status != -5:           # only HPT_ERR_BUSY (the bounded queue is full) is expected
                raise
            rejected += 1
    reap(True)
    if not done:
        return {"requests": len(requests), "rejected": rejected, "offered_rate_per_s": rate}
    times = np.array([t for t, _ in done]) / 1e6
    rs = [r for _, r in done]
    lat = times[:, 2] - times[:, 0]
    queue = times[:, 1] - times[:, 0]
    span = times[:, 2].max() - times[:, 0].min()
    by_size = {}
    for (W, H) in sorted({(r.W, r.H) for r in rs}):
        l = lat[[k for k, r in enumerate(rs) if (r.W, r.H) == (W, H)]]
        by_size[f"{W}x{H}"] = {"completed": int(len(l)), "p50_latency_s": float(np.percentile(l, 50)),
                               "p99_latency_s": float(np.percentile(l, 99))}
    return {"requests": len(requests), "rejected": rejected, "completed": len(done), "offered_rate_per_s": rate,
            "completed_rate_per_s": len(done) / span, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "max_latency_s": float(lat.max()),
            "p50_queue_s": float(np.percentile(queue, 50)), "p99_queue_s": float(np.percentile(queue, 99)),
            "holograms_per_s": sum(r.K for r in rs) / span,
            "path_samples_per_s": sum(r.path_samples() for r in rs) / span, "span_s": float(span),
            "latency_by_slm": by_size}


CFG4_DESC = ("Poisson arrivals; workload drawn uniformly from configs 0-3 (scenes of 4, 23k and 185k triangles, the "
             "185k-triangle scene with its 128^3 ambient cache; each config's pitch, wavelengths and depth), SLM "
             "512x512 / 1920x1080 / 3840x2160, spp in {16,32,64,128,256}, K in {1,4,8}, eye offsets U[-5,5] mm, "
             "focal depth U[5,30] mm; scenes and cache resident; outputs allocated by the library at admission")


def cfg4_context(hpt, S, device, max_inflight=8, max_queue=8):
    ctx = hpt.Context(device, max_inflight=max_inflight, max_queue=max_queue)
    sids = {"cfg0": ctx.upload_scene(S.config0_scene()), "cfg1": ctx.upload_scene(S.config1_scene()),
            "cfg3": ctx.upload_scene(S.config3_scene())}
    return ctx, sids


def run_serving(ctx, hpt, S, sid_cfg1, batched_holos, plain_holos, n_cfg4=2000):
    """(a) the headline request (1080p RGB 64 spp depth 4 K=8) offered above the device's capacity:
    the served throughput beside the batched and plain forms; (b) the serving workload of config 4:
    a seeded stream of n_cfg4 requests at 40 req/s with bounded admission (8 requests on the
    device, 8 waiting; a submission beyond that is rejected and counted)."""
    head = [(sid_cfg1, S.config2_render(seed=10 + k)) for k in range(12)]
    a = serve_owned(ctx, hpt, head, 8.0, 7)
    a["workload"] = "12 requests of the headline render (1920x1080 RGB, 64 spp, depth 4, K=8), Poisson 8 req/s"
    a["batched_holograms_per_s"] = batched_holos
    a["plain_fp64_holograms_per_s"] = plain_holos
    ctx.sync()
    bctx, sids = cfg4_context(hpt, S, ctx.device)
    try:
        reqs = [(sids[key], r) for key, r in S.config4_requests(n_cfg4, 4242)]
        b = serve_owned(bctx, hpt, reqs, 40.0, 8)
        b.update({"max_inflight": 8, "max_queue": 8, "workload": f"{n_cfg4} requests at 40 req/s, " + CFG4_DESC})
        bctx.sync()
    finally:
        bctx.close()
    return {"headline_at_capacity": a, "cfg4": b}


def run_serving_sweep(hpt, S, device, n, rates):
    """The config-4 stream with bounded admission at increasing offered rates: the highest rate
    sustained is the highest with no rejection and a p99 wait for admission under 1 s."""
    ctx, sids = cfg4_context(hpt, S, device)
    sweep, best = [], 0.0
    try:
        for k, rate in enumerate(rates):
            reqs = [(sids[key], r) for key, r in S.config4_requests(n, 5000 + k)]
            res = serve_owned(ctx, hpt, reqs, rate, 9 + k)
            sweep.append(res)
            if res["rejected"] == 0 and res.get("p99_queue_s", 1e9) <= 1.0:
                best = max(best, rate)
        ctx.sync()
    finally:
        ctx.close()
    return {"max_inflight": 8, "max_queue": 8, "requests_per_rate": n, "workload": CFG4_DESC, "rates": sweep,
            "max_sustained_rate_per_s": best}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, steps = bounded pixel samples."""
    from paper_2606_14173_gb300 import scenes as S
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl_desc, scene_fn, (render_fn, wl_over) = WORKLOADS[args.workload]
    sc = getattr(S, scene_fn)()
    r = getattr(S, render_fn)(**wl_over)
    n_pix = 2048 if args.workload != "cfg3" else 256
    for _ in range(args.warmup):
        cpu_oracle_rate(sc, r, max(n_pix // 8, 16))[0]
    rates, dts, samples = [], [], 0
    for k in range(args.steps):
        rate, dt, cores, ns = cpu_oracle_rate(sc, r, n_pix, seed=100 + k)[:4]
        dts.append(dt)
        samples += ns
    total = sum(dts)
    value = samples / total
    sample = (f"{n_pix} seeded random pixels of the {r.W}x{r.H} frame per step, {len(r.lambdas)} wavelengths, "
              f"{r.spp} spp, K={r.K}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_desc, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2606_14173_gb300 import build as pbuild, hpt, scenes as S

    if args.serving_sweep:
        pbuild.build()
        res = run_serving_sweep(hpt, S, 0, args.sweep_requests, [float(x) for x in args.serving_sweep.split(",")])
        print(json.dumps({"serving_sweep": res}), flush=True)
        return
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        pbuild.build()
    barrier(world)
    ctx = hpt.Context(local)
    wl_desc, scene_fn, (render_fn, wl_over) = WORKLOADS[args.workload]
    sc = getattr(S, scene_fn)()
    sid = ctx.upload_scene(sc)
    make_render = getattr(S, render_fn)
    r = make_render(seed=replica_seed(rank), **wl_over)
    samples_per_step = r.path_samples()
    # launch shape (wave size, lanes, grid sizes) chosen by the library's autotuner on a band of
    # this render, before any timing; kept for the scene's size class
    tuning = None if args.no_autotune else ctx.autotune(sid, r, precision=hpt.PREC_DF32)
    out = hpt.alloc_output(r)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    # all work on one dedicated stream: the legacy default stream serialises with the library's
    # wave stream and would add idle time between steps
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def step_mixed():
        ctx.trace(sid, r, out, precision=hpt.PREC_DF32, stream=stream)

    r_plain = [make_render(seed=replica_seed(rank), lambdas=(l,), channels=(c,), **wl_over)
               for l, c in zip(r.lambdas, r.channels)]
    outs_plain = [hpt.alloc_output(rp) for rp in r_plain]

    def step_plain():
        for rp, op in zip(r_plain, outs_plain):
            ctx.trace(sid, rp, op, precision=hpt.PREC_FP64, stream=stream)

    def timed(step, k, w, sample_clocks=False):
        clk = ClockSampler(local)
        if sample_clocks:
            clk.start()
            clk.wait_ready()
        for _ in range(w):
            flush.zero_()        # also loads the flush kernel before the timed region
            step()
        ctx.sync()
        barrier(world)
        torch.cuda.synchronize()
        th0 = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * k)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(k):
            flush.zero_()
            ev[2 * i].record(stream)
            step()
            ev[2 * i + 1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        th1 = time.perf_counter()
        barrier(world)
        clk.window(th0, th1)
        clocks = clk.stop() if sample_clocks else None
        ctx.sync()
        total_ms = t0.elapsed_time(t1)
        launch_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(k)]
        gaps = [t0.elapsed_time(ev[0])] + [ev[2 * i + 1].elapsed_time(ev[2 * i + 2]) for i in range(k - 1)]
        gaps_ms.append(gaps + [ev[2 * k - 1].elapsed_time(t1)])
        return allreduce_max(total_ms, world), launch_ms, clocks

    gaps_ms = []

    total_ms, launch_ms, clocks = timed(step_mixed, args.steps, args.warmup, sample_clocks=True)
    value = job_value(samples_per_step, args.steps, total_ms, world)
    holo_per_s = world * r.K * args.steps / (total_ms / 1e3)

    plain = None
    if not args.no_plain:
        pm, plm, _ = timed(step_plain, max(2, args.steps // 2), 1)
        kp = max(2, args.steps // 2)
        plain = {"value": world * samples_per_step * kp / (pm / 1e3), "unit": UNIT,
                 "holograms_per_s": world * r.K * kp / (pm / 1e3), "ms_per_step": pm / kp,
                 "form": "FP64 coherent arithmetic, one launch per wavelength (3 per step), K=8 path reuse"}

    # end to end through the public API with host memory: result copied to pinned host memory
    e2e = None
    if not args.no_e2e:
        host = torch.empty(tuple(out.shape), dtype=torch.complex64, pin_memory=True).numpy()
        for _ in range(max(1, args.warmup)):
            ctx.trace_host(sid, r, host, precision=hpt.PREC_DF32, stream=stream)
        barrier(world)
        t0 = time.perf_counter()
        k_e2e = max(3, args.steps)
        for _ in range(k_e2e):
            ctx.trace_host(sid, r, host, precision=hpt.PREC_DF32, stream=stream)
        e2e_s = allreduce_max(time.perf_counter() - t0, world)
        import ctypes
        h2d = ctypes.sizeof(hpt.RenderDesc)   # the render descriptor, copied to the device per call
        e2e = {"value": world * samples_per_step * k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(host.nbytes),
               "api": "hpt_trace_host (device trace; the rows each wave completes copied into pinned host memory "
                      "while later waves run, all K x 3 fields per step)"}

    # roofline of the dominant kernel (k_trace): its algorithmic FP32 work per frame from the work
    # counters, over its own device time per frame from CUDA events around every launch
    if args.no_counters:
        cnt = {"samples": 1, "box_tests": 0, "tri_tests": 0, "refines": 0, "shadow_rays": 0, "bounces": 0}
        kt = {k: (1.0, 1) for k in hpt.KERNEL_NAMES}
    else:
        cnt = ctx.trace_counters(sid, r, out, precision=hpt.PREC_DF32)
        kt = ctx.trace_timed(sid, r, out, precision=hpt.PREC_DF32)
    ns = max(cnt["samples"], 1)
    vertices = cnt["shadow_rays"] + cnt["bounces"] + cnt["refines"]
    trace_flops = (cnt["box_tests"] * FLOP_PER["box_tests"] + cnt["tri_tests"] * FLOP_PER["tri_tests"]
                   + cnt["refines"] * FLOP_PER["refines"])
    flops = trace_flops + vertices * FLOP_PER["vertex"] + ns * r.K * FLOP_PER["hologram"]
    trace_ms, trace_launches = kt["k_trace"]
    achieved = trace_flops / (trace_ms / 1e3) / 1e12
    kern_total = sum(ms for ms, _ in kt.values())
    traffic = TRACE_DRAM_BYTES_PER_LAUNCH if args.workload in ("cfg2", "band") else None
    probes = ctx.probe_peaks() if not args.no_counters else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / ALU_PEAK_TFLOPS, "traffic": traffic,
                "traffic_source": ("ncu capture of both trace kernels on the 1920x270 band with 2M-path waves, "
                                   "scaled x4.0 to the 8M-path waves of this frame" if traffic is not None else None),
                "kernel": "k_trace",
                "issue": TRACE_ISSUE if args.workload in ("cfg2", "band") else None,
                "issue_source": ("ncu --set full capture of each trace kernel on the 1920x270 band with "
                                 "2M-path waves" if args.workload in ("cfg2", "band") else None),
                "measured_probes": probes,
                "frac_of_measured_fp32": (achieved / probes["fp32_tflops"]) if probes else None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz (no measured FP32 peak)",
                "launches_per_frame": trace_launches, "ms_per_launch": trace_ms / max(trace_launches, 1),
                "flop_per_launch": trace_flops / max(trace_launches, 1),
                "kernel_share": {k: ms / kern_total for k, (ms, _) in kt.items()},
                "whole_path_tflops": flops / statistics.mean([x / 1e3 for x in launch_ms]) / 1e12,
                "per_sample": {k: v / ns for k, v in cnt.items() if k != "samples"},
                "flops_per_sample": flops / ns}

    optics = None
    if not args.no_optics and rank == 0:
        optics = run_optics(ctx, hpt, torch, r, out, sid, stream)
        ctx.sync()

    serving = None
    if not args.no_serving and args.workload == "cfg2" and rank == 0:
        serving = run_serving(ctx, hpt, S, sid, holo_per_s, plain["holograms_per_s"] if plain else None,
                              args.cfg4_requests)
        ctx.sync()

    cpu = None
    precision = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        npx = 8192 if args.workload != "cfg3" else 1024
        # the fields of both forms, traced once more outside the timing (later measurements reuse
        # the buffers), for the error report against the oracle's pixels
        ctx.trace(sid, r, out, precision=hpt.PREC_DF32, stream=stream)
        if not args.no_plain:
            step_plain()
        ctx.sync()
        torch.cuda.synchronize()
        rate, dt, cores, nsamp, pix, ref = cpu_oracle_rate(sc, r, npx)
        pix_t = torch.from_numpy(np.asarray(pix)).to(out.device)
        U_df = out.reshape(out.shape[0], out.shape[1], -1)[:, :, pix_t].cpu().numpy()
        import oracle
        orc = oracle.Oracle(sc)
        pix_np = np.asarray(pix)

        def flags_df(sel):
            _, fl, sv = orc.trace(r, pix_np[sel], with_flags=True)
            return fl, sv
        precision = {"df32": precision_report(U_df, ref, flags_df)}
        if not args.no_plain:
            # the plain form renders each wavelength on its own (wavelength index 0 in the draws):
            # its reference is the oracle on those single-wavelength renders
            U_64 = np.stack([o.reshape(o.shape[1], -1)[:, pix_t].cpu().numpy() for o in outs_plain])
            ref_64 = np.concatenate([orc.trace(rp, pix_np) for rp in r_plain])

            def flags_64(sel):
                res = [orc.trace(rp, pix_np[sel], with_flags=True) for rp in r_plain]
                return np.concatenate([x[1] for x in res]), np.concatenate([x[2] for x in res])
            precision["fp64"] = precision_report(U_64, ref_64, flags_64)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{npx} seeded random pixels of the {r.W}x{r.H} frame x {len(r.lambdas)} wavelengths x "
                         f"{r.spp} spp ({nsamp} path samples, {dt:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
                "config": {"workload": wl_desc,
                           "path_samples_per_step": samples_per_step, "parallelism": f"replicas x{world}",
                           "l2": "flushed between steps (256 MiB write)"},
                "holograms_per_s": holo_per_s, "plain_fp64": plain, "launch_ms": launch_ms,
                "idle_ms_per_step": (total_ms - sum(launch_ms)) / args.steps,
                "gaps_ms": [round(g, 3) for g in gaps_ms[0]],
                "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps * sum(n for _, n in kt.values()),
                "graph_launches": args.steps, "autotune": tuning, "roofline": roofline, "optics": optics, "serving": serving, "precision": precision,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
