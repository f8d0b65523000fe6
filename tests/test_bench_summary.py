"""bench.py's reporting helpers on CPU: the compact summary survives legs
that failed (each reports its error instead of ending the run), the parity
accumulator measures what it states, and the tick-trace digest of the
serving legs reads a trace record array."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_summary_survives_failed_legs():
    line = {"value": 2.5e10, "roofline": {"frac": 0.03}, "step_roofline": {"frac": 0.07},
            "e2e": {"error": "RuntimeError: x"}, "other_workloads": {"error": "y"},
            "serving": {"error": "z"}, "serving_mixed": None, "parity": {"error": "w"}}
    s = bench.summary(line)
    assert s["Gev_s"][bench.HEADLINE] == 25.0
    assert s["e2e_Gev_s"] is None and s["e2e_events16_Gev_s"] is None
    assert s["serving"] == {"c3": {"error": "z"}}
    assert s["parity(err,err1e-3C,ulpsC,lsb,off,frames)"] == {}


def test_parity_accumulator():
    acc = bench.ParityAcc()
    C = 0.25
    ref = np.array([0.0, 0.5, -0.125, 1.0])
    got = ref.astype(np.float32).copy()
    got[0] = np.float32(3 * np.spacing(np.float32(C)))    # 3 ulps of C near zero
    got[1] = np.float32(0.5 + 1e-6)
    acc.state(got, np.arange(4), ref, np.arange(4), C)
    a = np.zeros((2, 3, 4), np.uint8)
    b = a.copy()
    b[1, 2, 3] = 1
    acc.frames_(a, b)
    out = acc.out()
    assert abs(out["abs_err_near_zero_ulps_of_C"] - 3.0) < 1e-6
    assert abs(out["state_err"] - float(np.float32(0.5 + 1e-6) - 0.5) / 0.5) < 1e-9
    assert out["T_exact"] and out["frame_max_lsb"] == 1 and out["frame_off_by_one"] == 1
    assert out["frames"] == 2 and out["pass"]
    acc.state(got, np.arange(4) + 1, ref, np.arange(4), C)
    assert not acc.out()["T_exact"] and not acc.out()["pass"]


class _FakeEsi:
    def __init__(self, tr):
        self.tr = tr

    def esi_server_trace(self, srv):
        return 0, self.tr


def test_tick_digest():
    dt = np.dtype([("call_ns", np.int64), ("issued_ns", np.int64), ("ready_ns", np.int64),
                   ("copy_ms", np.float32), ("kernels_ms", np.float32), ("gap_ms", np.float32),
                   ("frames", np.int32), ("events", np.int64), ("streams", np.int32),
                   ("items", np.int32)], align=True)
    tr = np.zeros(6, dt)
    tr["call_ns"] = [0, 1_000_000, 2_000_000, 5_000_000, 6_000_000, 7_000_000]   # one 3 ms gap
    tr["issued_ns"] = tr["call_ns"] + 40_000
    tr["ready_ns"] = tr["call_ns"] + 150_000
    tr["kernels_ms"] = 0.1
    tr["gap_ms"] = [-1, 0.5, 0.001, 2.0, 0.0, 0.7]                # two ticks queued behind another
    tr["frames"] = [0, 2, 3, 1, 4, 0]
    d = bench._tick_gaps(_FakeEsi(tr), None)
    assert d["max_tick_gap_ms"] == 3.0 and d["tick_gaps_over_2ms"] == 1 and d["traced_ticks"] == 6
    f = d["frame_ticks_ms(p50,p99)"]
    assert f["host"] == [0.04, 0.04] and f["call_to_ready"] == [0.15, 0.15]
    assert f["queued_share"] == 0.5
    assert bench._tick_gaps(_FakeEsi(tr[:1]), None) == {}
