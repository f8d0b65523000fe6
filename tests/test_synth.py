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


def test_sinusoid_short_is_deterministic_and_ordered():
    sc = synth.sinusoid_346x260(duration_s=0.1, t0_us=5000)
    a = synth.generate(sc, threads=1)
    b = synth.generate(sc, threads=4)
    assert len(a) > 50_000
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    _check_stream(a, sc)


def test_blobs_small_sensor():
    sc = synth.blobs_640x480(duration_s=0.2, W=96, H=64, n_blobs=6)
    ev = synth.generate(sc)
    assert len(ev) > 1000
    _check_stream(ev, sc)
    # per-pixel thresholds differ, so both polarities appear
    assert (ev["p"] > 0).mean() > 0.2 and (ev["p"] < 0).mean() > 0.2


def test_checkerboard_small_sensor_has_hot_pixels_and_bursts():
    sc = synth.checkerboard_1280x720(duration_s=0.4, W=160, H=96)
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


def _keys(ev):
    return set(zip(ev["t"].tolist(), ev["x"].tolist(), ev["y"].tolist(), ev["p"].tolist()))


def test_thinning_keeps_a_subset_at_the_asked_fraction():
    sc = synth.blobs_640x480(duration_s=0.05, W=160, H=120, n_blobs=10)
    full = synth.generate(sc)
    sc.keep_prob = 0.3
    thin = synth.generate(sc)
    assert np.all(np.diff(thin["t"]) >= 0)
    # the thinning draws come from their own generator: the kept events are
    # exactly events of the unthinned stream
    assert _keys(thin) <= _keys(full)
    frac = len(thin) / len(full)
    assert abs(frac - 0.3) < 4 * np.sqrt(0.3 * 0.7 / len(full)) + 0.01, frac


def test_mixed_serving_workload_shape():
    ws = synth.mixed_serving(duration_s=0.1)
    assert len(ws) == 192
    dims = [(w["W"], w["H"]) for w in ws]
    assert dims.count((1280, 720)) == 16 and dims.count((640, 480)) == 48
    assert dims.count((346, 260)) == 128
    assert sum(W * H for W, H in dims) == 41_006_080
    for w in ws:
        assert 0.1e6 <= w["rate"] <= 20e6
        assert w["t_join_us"] % 1000 == 0 and 0 <= w["t_join_us"] < 50_000
        if w["t_leave_us"] is not None:
            assert w["t_leave_us"] % 1000 == 0 and 50_000 <= w["t_leave_us"] < 100_000
        assert w["scene"].t0_us == w["t_join_us"]
    assert any(w["t_join_us"] > 0 for w in ws) and any(w["t_leave_us"] for w in ws)
    # deterministic
    again = synth.mixed_serving(duration_s=0.1)
    assert [(w["rate"], w["t_join_us"], w["t_leave_us"]) for w in again] == \
        [(w["rate"], w["t_join_us"], w["t_leave_us"]) for w in ws]


def test_pack_events_layout():
    ev = np.zeros(3, dtype=synth.EVENT_DTYPE)
    ev["t"] = [100, 101, 100 + 2**31 - 1]
    ev["x"] = [5, 65535, 0]
    ev["y"] = [7, 65535, 1]
    ev["p"] = [1, -1, 0]
    w = synth.pack_events(ev, 100)
    assert w.dtype == np.uint64
    assert int(w[0]) == 5 + 7 * 2**16 + 2**32
    assert int(w[1]) == 65535 + 65535 * 2**16 + 1 * 2**33
    assert int(w[2]) == 2**16 + (2**31 - 1) * 2**33
    import pytest
    with pytest.raises(ValueError):
        synth.pack_events(ev, 101)           # a time before the base
    with pytest.raises(ValueError):
        synth.pack_events(ev, 99)            # an offset of 2^31
