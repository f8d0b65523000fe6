"""The seeded generator produces valid, deterministic, time-ordered streams."""
import numpy as np

import synth


def _check_stream(ev, sc):
    assert ev.dtype == synth.EVENT_DTYPE
    assert np.all(np.diff(ev["t"]) >= 0)
    assert np.all(ev["x"] < sc.W) and np.all(ev["y"] < sc.H)
    assert set(np.unique(ev["p"]).tolist()) <= {-1, 1}
    assert ev["t"].min() >= sc.t0_us
    assert ev["t"].max() <= sc.t0_us + int(round(sc.duration_s * 1e6))
    # ties in t are ordered by pixel index
    pix = ev["y"].astype(np.int64) * sc.W + ev["x"]
    same = np.diff(ev["t"]) == 0
    assert np.all(np.diff(pix)[same] >= 0)


def test_config0_short_is_deterministic_and_ordered():
    sc = synth.config0(duration_s=0.1, t0_us=5000)
    a = synth.generate(sc, threads=1)
    b = synth.generate(sc, threads=4)
    assert len(a) > 50_000
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    _check_stream(a, sc)


def test_config1_small_sensor():
    sc = synth.config1(duration_s=0.2, W=96, H=64, n_blobs=6)
    ev = synth.generate(sc)
    assert len(ev) > 1000
    _check_stream(ev, sc)
    # per-pixel thresholds differ, so both polarities appear
    assert (ev["p"] > 0).mean() > 0.2 and (ev["p"] < 0).mean() > 0.2


def test_config2_small_sensor_has_hot_pixels_and_bursts():
    sc = synth.config2(duration_s=0.4, W=160, H=96)
    sc.hot_frac = 0.01
    ev = synth.generate(sc)
    _check_stream(ev, sc)
    cnt = np.bincount(ev["y"].astype(np.int64) * sc.W + ev["x"], minlength=sc.W * sc.H)
    assert cnt.max() > 50 * np.median(cnt[cnt > 0])     # heavy tail (hot pixels)
    per_ms = np.bincount(ev["t"] // 1000, minlength=400)
    assert per_ms[300:340].mean() > 2 * np.median(per_ms)  # flicker burst


def test_serving_stream_rate():
    sc = synth.serving_stream(3, 2.0e6, 0.05)
    ev = synth.generate(sc)
    rate = len(ev) / 0.05
    assert 1.0e6 < rate < 3.0e6
