"""bench.py's end-to-end leg on CPU, against a fake library that records
every call: each step pushes exactly its own events (16-byte events with
shifted times, or the packed words with a shifted time base) and renders
exactly its own frames, steps follow one another with no gap or repeat
across runs and input kinds, a packed run covers max(3, min(steps, 30)) steps, and the
reported rates and byte counts follow from them."""
import os
import sys
import types

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


class _FakeTorch:
    uint8 = torch.uint8

    @staticmethod
    def empty(shape, dtype=None, pin_memory=False):
        return torch.empty(shape, dtype=dtype)


class _FakeEsi:
    def __init__(self, ev, span, win, M):
        self.ev, self.span, self.win, self.M = ev, span, win, M
        self.t0 = int(ev["t"][0])
        self.words = synth.pack_events(ev, self.t0)
        self.steps = []          # (step index, packed) per push
        self.rendered = []       # step index per render
        self.syncs = 0

    @staticmethod
    def check(rc, what=""):
        if rc:
            raise RuntimeError(f"{what}: {rc}")

    def esi_push_packed(self, h, buf, n, t_base, on_device):
        assert on_device == 0 and n == len(self.ev)
        assert np.array_equal(buf.numpy().view(np.uint64), self.words)
        k, rem = divmod(t_base - self.t0, self.span)
        assert rem == 0
        self.steps.append((k, True))
        return 0

    def esi_push_events(self, h, buf, n, on_device):
        assert on_device == 0 and n == len(self.ev)
        got = buf.numpy().view(self.ev.dtype)
        k, rem = divmod(int(got["t"][0]) - int(self.ev["t"][0]), self.span)
        assert rem == 0
        assert np.array_equal(got["t"], self.ev["t"] + k * self.span)
        assert np.array_equal(got["x"], self.ev["x"]) and np.array_equal(got["p"], self.ev["p"])
        self.steps.append((k, False))
        return 0

    def esi_render_frames(self, h, tf, m, out, mode):
        assert m == self.M and mode in (0, 2) and tuple(out.shape) == (self.M, 3, 4)
        k = self.steps[-1][0]
        assert np.array_equal(tf, bench.frame_times(k, self.span, self.win))
        self.rendered.append(k)
        return 0

    def esi_synchronize(self, h):
        self.syncs += 1
        return 0

    def esi_get_stats(self, h):
        return 0, types.SimpleNamespace(ring_capacity=1 << 20, ring_grows=0, push_waits=0)


@pytest.mark.parametrize("steps", [1, 3, 7, 45])
def test_e2e_leg_steps_are_consecutive_and_counted(steps, monkeypatch):
    span, win = 10_000, 1_000
    M = span // win
    ev = np.zeros(50, dtype=synth.EVENT_DTYPE)
    ev["t"] = 5 + np.sort(np.random.default_rng(0).integers(0, span, 50))
    ev["x"], ev["y"], ev["p"] = np.arange(50) % 4, np.arange(50) % 3, 1 - 2 * (np.arange(50) % 2)
    fake = _FakeEsi(ev, span, win, M)
    clock = iter(np.arange(0, 1e6, 0.5))       # every run takes 0.5 s per timer pair
    monkeypatch.setattr(bench.time, "perf_counter", lambda: next(clock))
    r = {"handle": object(), "ev": ev, "span": span, "win": win, "M": M,
         "sc": types.SimpleNamespace(W=4, H=3), "total": 8}
    out = bench.e2e_leg(fake, _FakeTorch, r, steps)

    ks = [k for k, _ in fake.steps]
    assert ks == list(range(8, 8 + len(ks)))             # no gap, no repeat
    assert fake.rendered == ks
    per_packed = max(3, min(steps, 30))
    n_packed = sum(1 for _, p in fake.steps if p)
    n_16 = len(fake.steps) - n_packed
    assert n_packed == per_packed * (2 + 5 + 5)          # 2 warm-up, 5 pipelined, 5 synchronous
    assert n_16 == 3 * (2 + 5 + 5)
    assert fake.syncs == 2 * (2 + 5 + 5)
    assert out["steps"] == out["steps_per_run"] == per_packed
    assert out["events16"]["steps_per_run"] == 3
    # each timed run spans one 0.5 s timer step
    assert out["value"] == pytest.approx(len(ev) * per_packed / 0.5)
    assert out["events16"]["value"] == pytest.approx(len(ev) * 3 / 0.5)
    assert out["h2d_bytes_per_step"] == len(ev) * 8
    assert out["events16"]["h2d_bytes_per_step"] == len(ev) * 16
    assert out["d2h_bytes_per_step"] == M * 4 * 3
    assert out["frames_per_s"] == pytest.approx(M * per_packed / 0.5)
