"""Host logic of the serving measurement (no GPU): Poisson submission with library-owned outputs,
BUSY answers counted as rejections, every completed request released once, latency and rate
statistics from the request timestamps."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Err(RuntimeError):
    def __init__(self, status):
        super().__init__(f"status {status}")
        self.status = status


class _FakeCtx:
    """Answers BUSY to every third submission; request k runs from 10 k ms to 10 k + 50 ms after
    an admission delay of 2 ms."""

    def __init__(self, fail_status=-5):
        self.n, self.accepted, self.fail_status, self.released = 0, [], fail_status, []

    def sync(self):
        pass

    def submit(self, sid, r, out, precision=1):
        assert out is None                      # outputs owned by the library
        self.n += 1
        if self.n % 3 == 0:
            raise _Err(self.fail_status)
        self.accepted.append(self.n)
        return self.n

    def poll(self, i):
        return i % 2 == 0                       # even ids finish early, odd ones need a wait

    def wait(self, i, timeout_ms):
        pass

    def request_release(self, i):
        assert i not in self.released
        self.released.append(i)

    def request_times(self, i):
        t0 = 10e3 * i
        return (t0, t0 + 2e3, t0 + 50e3)


def _requests(n):
    r = types.SimpleNamespace(K=4, W=64, H=32, path_samples=lambda: 1000)
    return [(1, r) for _ in range(n)]


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_busy_answers_are_counted_and_excluded(bench):
    ctx = _FakeCtx()
    res = bench.serve_owned(ctx, types.SimpleNamespace(HptError=_Err, PREC_DF32=1), _requests(9), 1e6, 0)
    assert res["requests"] == 9 and res["rejected"] == 3 and res["completed"] == 6
    assert sorted(ctx.released) == ctx.accepted
    ids = ctx.accepted                                   # 1, 2, 4, 5, 7, 8
    span = (10e3 * ids[-1] + 50e3 - 10e3 * ids[0]) / 1e6
    assert res["completed_rate_per_s"] == pytest.approx(6 / span)
    assert res["p50_latency_s"] == pytest.approx(0.05) and res["p99_latency_s"] == pytest.approx(0.05)
    assert res["p50_queue_s"] == pytest.approx(0.002) and res["p99_queue_s"] == pytest.approx(0.002)
    assert res["latency_by_slm"] == {"64x32": {"completed": 6, "p50_latency_s": pytest.approx(0.05),
                                                "p99_latency_s": pytest.approx(0.05)}}
    assert res["holograms_per_s"] == pytest.approx(6 * 4 / span)
    assert res["path_samples_per_s"] == pytest.approx(6 * 1000 / span)


def test_other_errors_are_not_swallowed(bench):
    hpt = types.SimpleNamespace(HptError=_Err, PREC_DF32=1)
    with pytest.raises(_Err):
        bench.serve_owned(_FakeCtx(fail_status=-1), hpt, _requests(4), 1e6, 0)


def test_all_rejected_gives_counts_only(bench):
    class AllBusy(_FakeCtx):
        def submit(self, *a, **k):
            raise _Err(-5)
    hpt = types.SimpleNamespace(HptError=_Err, PREC_DF32=1)
    res = bench.serve_owned(AllBusy(), hpt, _requests(3), 1e6, 0)
    assert res == {"requests": 3, "rejected": 3, "offered_rate_per_s": 1e6}


class _DoneProc:
    """Stands in for the nvidia-smi process once its samples are in."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clock_rows(samples):
    # (time, [index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap])
    return [(t, ["0", str(sm), "2070", "900.0", "0x0", hw, "Not Active", "Not Active", pc]) for t, sm, hw, pc in samples]


def test_clock_sampler_keeps_the_timed_window_and_reports_reasons(bench):
    """The bench's clock record: only samples inside the timed window count; the median SM clock,
    the maximum clock and every throttle reason seen active inside the window are reported."""
    clk = bench.ClockSampler(0)
    clk.proc = _DoneProc()
    clk.rows = _clock_rows([(0.0, 345, "Not Active", "Not Active"),      # start-up, outside the window
                            (1.0, 2070, "Not Active", "Not Active"),
                            (1.2, 2055, "Not Active", "Active"),
                            (1.4, 2070, "Not Active", "Not Active"),
                            (9.0, 900, "Active", "Not Active")])         # after the window
    clk.window(0.9, 1.5)
    rec = clk.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    clk.rows.append((1.3, ["0", "1500", "2070", "800", "0x8", "Active", "Not Active", "Not Active", "Not Active"]))
    clk.rows.append((1.35, ["0", "garbled"]))                             # a broken line is skipped
    rec = clk.stop()
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"] and rec["samples"] == 4


def test_clock_sampler_without_nvidia_smi(bench):
    clk = bench.ClockSampler(0)
    assert clk.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
