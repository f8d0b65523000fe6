"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Inputs come only from the seeded generator; expected values only from the
oracle.  Tolerances are defined in esi_harness (state 1e-5 relative with a
floor of C, T exact, frames within 1 LSB).
"""
import numpy as np
import pytest

import oracle
import synth
from esi_harness import (EXACT, GpuStream, compare, random_events, run_gpu, run_oracle,
                         state_error, STATE_TOL)

pytestmark = pytest.mark.gpu

BASE = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)


def P(**kw):
    d = dict(BASE)
    d.update(kw)
    return d


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


# ------------------------------------------------------------- small streams
SHAPES = [(37, 19), (100, 70), (346, 260), (64, 64)]


@pytest.mark.parametrize("W,H", SHAPES)
@pytest.mark.parametrize("b,k", [(2.0, 10.0), (0.5, 100.0), (3.7, 1.0), (1.0, 0.0), (2.5, 1e4)])
@pytest.mark.parametrize("rd", [0, 1])
def test_random_stream_replay(W, H, b, k, rd):
    rng = np.random.default_rng(W * 131 + H + int(b * 10) + int(k) + rd)
    n = 20_000
    ev = random_events(rng, W, H, n, 0, 400_000)
    p = P(b=b, k_per_s=k, render_decay=rd, s_min=-0.8, s_max=1.2)
    tf = np.arange(10_000, 400_001, 10_000)
    ref = run_oracle(ev, W, H, p, tf)
    gpu = run_gpu(ev, W, H, p, tf)
    compare(gpu, ref, p["C"], f"{W}x{H} b={b} k={k} rd={rd}")


def test_per_frame_equals_replay_bitwise():
    rng = np.random.default_rng(3)
    W, H = 130, 90
    ev = random_events(rng, W, H, 50_000, 0, 1_000_000, hot=(5, 7, 0.05))
    p = P(render_decay=1)
    tf = np.arange(20_000, 1_000_001, 20_000)
    a = run_gpu(ev, W, H, p, tf, mode="replay", tuning=EXACT)
    b = run_gpu(ev, W, H, p, tf, mode="per_frame", tuning=EXACT)
    assert np.array_equal(a["S"], b["S"]) and np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["frames"], b["frames"])
    compare(a, run_oracle(ev, W, H, p, tf), p["C"])


TUNINGS = [
    dict(tile_h=4), dict(tile_h=8), dict(tile_h=16),
    dict(tile_w=32, tile_h=16), dict(tile_w=32, tile_h=32),
    dict(tile_w=64, tile_h=4), dict(tile_w=64, tile_h=8), dict(tile_w=64, tile_h=16),
    dict(tile_w=64, tile_h=8, batch_records=2048, chunk_events=1024),
    dict(tile_w=32, tile_h=32, batch_records=1024, chunk_events=512),
    dict(chunk_events=512), dict(chunk_events=8192),
    dict(batch_records=1024), dict(batch_records=8192),
    dict(max_batch_events=4096, chunk_events=512),
    dict(tile_h=8, chunk_events=1024, batch_records=1024, max_batch_events=3000),
]


def test_launch_shapes_give_bit_identical_results():
    # binning is exact, so every tile/chunk/batch shape applies each pixel's
    # events in the same order with the same arithmetic (the scan off: it
    # rounds each group's composition its own way)
    rng = np.random.default_rng(4)
    W, H = 200, 150
    ev = random_events(rng, W, H, 80_000, 0, 800_000, hot=(33, 40, 0.1))
    p = P(render_decay=1, b=1.7)
    tf = np.arange(10_000, 800_001, 10_000)
    ref = run_gpu(ev, W, H, p, tf, tuning=EXACT)
    compare(ref, run_oracle(ev, W, H, p, tf), p["C"])
    for t in TUNINGS:
        g = run_gpu(ev, W, H, p, tf, tuning={**t, **EXACT})
        assert np.array_equal(g["S"], ref["S"]), t
        assert np.array_equal(g["T"], ref["T"]), t
        assert np.array_equal(g["frames"], ref["frames"]), t


# ------------------------------------------------------------- the workloads
@pytest.fixture(scope="module")
def scene_streams():
    return {}


def _scene(scene_streams, make):
    """The full-size stream of a scene generator, generated once per module."""
    if make not in scene_streams:
        sc = make()
        scene_streams[make] = (sc, synth.generate(sc))
    return scene_streams[make]


# contrast step C of each scene (its generator's mean threshold)
SCENE_C = {synth.sinusoid_346x260: 0.2, synth.blobs_640x480: 0.15,
           synth.checkerboard_1280x720: 0.2}


@pytest.mark.parametrize("rd", [0, 1])
def test_sinusoid_346x260_full(scene_streams, rd):
    sc, ev = _scene(scene_streams, synth.sinusoid_346x260)
    p = P(C=SCENE_C[synth.sinusoid_346x260], render_decay=rd)
    tf = np.arange(10_000, 1_000_001, 10_000)
    res = compare(run_gpu(ev, sc.W, sc.H, p, tf), run_oracle(ev, sc.W, sc.H, p, tf), p["C"],
                  "sinusoid 346x260")
    print("sinusoid 346x260", rd, res)


def test_blobs_640x480_full(scene_streams):
    sc, ev = _scene(scene_streams, synth.blobs_640x480)
    p = P(C=SCENE_C[synth.blobs_640x480], render_decay=1)
    tf = np.arange(10_000, 2_000_001, 10_000)
    res = compare(run_gpu(ev, sc.W, sc.H, p, tf), run_oracle(ev, sc.W, sc.H, p, tf), p["C"],
                  "blobs 640x480")
    print("blobs 640x480", res)


def test_checkerboard_1280x720_full_10ms(scene_streams):
    sc, ev = _scene(scene_streams, synth.checkerboard_1280x720)
    p = P(C=SCENE_C[synth.checkerboard_1280x720], render_decay=1)
    tf = np.arange(10_000, 1_000_001, 10_000)
    res = compare(run_gpu(ev, sc.W, sc.H, p, tf), run_oracle(ev, sc.W, sc.H, p, tf), p["C"],
                  "checkerboard 1280x720")
    print("checkerboard 1280x720", res)


def test_checkerboard_1280x720_1ms_windows_sampled(scene_streams):
    # 1000 frames of 1280x720: compare the final state in full and a sample of
    # frames the oracle renders one by one (frames never change the state)
    import torch
    sc, ev = _scene(scene_streams, synth.checkerboard_1280x720)
    p = P(C=SCENE_C[synth.checkerboard_1280x720], render_decay=1)
    tf = np.arange(1_000, 1_000_001, 1_000)
    with GpuStream(sc.W, sc.H, p) as g:
        assert g.push(ev) == 0
        out = torch.empty((len(tf), sc.H, sc.W), dtype=torch.uint8, device="cuda")
        assert g.esi.esi_render_frames(g.h, tf, len(tf), out, 1) == 0
        assert g.esi.esi_synchronize(g.h) == 0
        S, T = g.state()
        sample = [0, 1, 299, 300, 305, 317, 500, 701, 702, 998, 999]
        frames = out[sample].cpu().numpy()
    st = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**{k: p[k] for k in BASE}, render_decay=1))
    ref_frames = []
    i = 0
    for w in sample:
        j = int(np.searchsorted(ev["t"], tf[w], side="right"))
        st.integrate(ev[i:j])
        i = j
        ref_frames.append(st.render(tf[w]))
    st.integrate(ev[i:])
    res = compare({"S": S, "T": T, "frames": frames},
                  {"S": st.S, "T": st.T, "frames": np.stack(ref_frames)}, p["C"], "checkerboard 1280x720, 1 ms")
    print("checkerboard 1280x720, 1 ms", res)


# ---------------------------------------------------------------- edge cases
def test_no_events_frames_and_state():
    p = P(t_origin_us=500, s_min=-0.5, s_max=1.5, render_decay=1)
    W, H = 50, 33
    with GpuStream(W, H, p) as g:
        rc, fr = g.render_frames([500, 1000, 10**9])
        assert rc == 0
        assert np.all(fr == 64)      # 255 * 0.5 / 2 = 63.75 -> 64
        S, T = g.state()
        assert np.all(S == 0) and np.all(T == 500)


def test_single_event_and_cutoff():
    # C = 0.5, k = 1e5/s (0.1 per us), b = 2: an event 5 us after the origin
    # contributes 0.5 * 0.25; one 11 us after contributes 0 (Eq. 4 cutoff)
    p = P(C=0.5, k_per_s=1e5, b=2.0)
    ev = random_events(np.random.default_rng(0), 4, 4, 2, 0, 1)
    ev["t"] = [5, 11]
    ev["x"] = [1, 2]
    ev["y"] = [1, 3]
    ev["p"] = [1, -1]
    g = run_gpu(ev, 4, 4, p, [20])
    S = g["S"].reshape(4, 4)
    assert S[1, 1] == pytest.approx(0.125, rel=1e-6)
    assert S[3, 2] == 0.0
    compare(g, run_oracle(ev, 4, 4, p, [20]), p["C"])


def test_event_at_frame_time_is_included_and_later_ones_wait():
    p = P(C=0.5, k_per_s=0.0)
    ev = random_events(np.random.default_rng(0), 2, 1, 3, 0, 1)
    ev["t"] = [100, 200, 201]
    ev["x"] = [0, 0, 1]
    ev["y"] = 0
    ev["p"] = 1
    with GpuStream(2, 1, p) as g:
        assert g.push(ev) == 0
        rc, fr = g.render_frame(200)
        assert rc == 0
        S, _ = g.state()
        assert S[0] == 1.0 and S[1] == 0.0          # t = 200 in, t = 201 pending
        assert g.stats().events_pending == 1
        rc, fr = g.render_frame(201)
        S, T = g.state()
        assert S[1] == 0.5 and T[1] == 201


def test_ties_same_pixel_same_time_keep_arrival_order():
    # order only matters through the clamp: (+, +, -) vs (-, +, +) at one time
    p = P(C=0.6, k_per_s=1e5, b=1.0, s_min=-1.0, s_max=1.0)
    for pols in ([1, 1, -1], [-1, 1, 1], [1, -1, 1]):
        ev = random_events(np.random.default_rng(0), 3, 3, 3, 0, 1)
        ev["t"] = 5
        ev["x"] = 1
        ev["y"] = 2
        ev["p"] = pols
        g = run_gpu(ev, 3, 3, p, [5])
        compare(g, run_oracle(ev, 3, 3, p, [5]), p["C"], str(pols))


def test_out_of_range_events_are_dropped_and_counted():
    rng = np.random.default_rng(8)
    W, H = 40, 30
    ev = random_events(rng, W + 5, H + 5, 5000, 0, 100_000)
    p = P()
    g = run_gpu(ev, W, H, p, [100_000])
    ref = run_oracle(ev, W, H, p, [100_000])
    assert g["dropped"] == ref["dropped"] > 0
    compare(g, ref, p["C"])


def test_time_order_violations_are_rejected_whole():
    p = P()
    ev = random_events(np.random.default_rng(1), 8, 8, 10, 0, 1000)
    with GpuStream(8, 8, p) as g:
        bad = ev.copy()
        bad["t"][5] = bad["t"][4] - 1
        assert g.push(bad) == g.esi.ESI_ETIMEORDER
        assert g.stats().events_pushed == 0
        assert g.push(bad, on_device=True) == g.esi.ESI_ETIMEORDER
        assert g.stats().events_pushed == 0
        assert g.push(ev) == 0
        late = ev[:1].copy()
        late["t"] = ev["t"][-1] - 1
        assert g.push(late) == g.esi.ESI_ETIMEORDER
        rc, _ = g.render_frame(2000)
        assert rc == 0
        rc, _ = g.render_frame(1999)
        assert rc == g.esi.ESI_ETIMEORDER
        early = ev[:1].copy()
        early["t"] = 1500
        assert g.push(early) == g.esi.ESI_ETIMEORDER   # before the last frame


def test_hot_pixel_spanning_many_batches():
    # one tile receives several shared-memory batches; one pixel holds most events
    rng = np.random.default_rng(12)
    W, H = 64, 40
    ev = random_events(rng, W, H, 60_000, 0, 3_000_000, hot=(10, 10, 0.5))
    p = P(C=0.05, k_per_s=2.0, b=3.7, render_decay=1)
    tf = np.arange(50_000, 3_000_001, 50_000)
    for t in (None, dict(batch_records=1024)):
        compare(run_gpu(ev, W, H, p, tf, tuning=t), run_oracle(ev, W, H, p, tf), p["C"], str(t))


def test_ring_wraps_across_many_pushes_and_renders():
    rng = np.random.default_rng(13)
    W, H = 96, 64
    n = 3_000_000                      # > the initial ring of 2^20 events
    ev = random_events(rng, W, H, n, 0, 30_000_000)
    p = P(render_decay=1)
    st = oracle.OracleState(W, H, oracle.OracleParams(**BASE, render_decay=1))
    with GpuStream(W, H, p) as g:
        pos = 0
        t = 0
        step = 250_000
        while pos < n:
            nxt = min(n, pos + 600_000)
            assert g.push(ev[pos:nxt]) == 0
            pos = nxt
            t_hi = int(ev["t"][pos - 1]) - 1 if pos < n else 30_000_000
            tfs = np.arange(t + step, t_hi, step)
            if len(tfs):
                rc, fr = g.render_frames(tfs)
                assert rc == 0
                ref_fr, _ = st.replay(ev[np.searchsorted(ev["t"], t, "right"):], tfs)
                d = np.abs(fr.astype(int) - ref_fr.astype(int)).max()
                assert d <= 1
                t = int(tfs[-1])
        rc, _ = g.render_frame(30_000_000)
        assert rc == 0
        st.integrate(ev[np.searchsorted(ev["t"], t, "right"):])
        S, T = g.state()
    assert state_error(S, st.S, p["C"]) <= STATE_TOL
    assert np.array_equal(T, st.T)


def test_time_span_beyond_32_bits_is_split():
    # events hours apart: record times are 32-bit offsets, so the render splits
    rng = np.random.default_rng(14)
    W, H = 33, 17
    ev = random_events(rng, W, H, 4000, 0, 3 * 2**32)
    p = P(k_per_s=1e-4, b=1.5)
    tf = np.linspace(2**31, 3 * 2**32, 7).astype(np.int64)
    compare(run_gpu(ev, W, H, p, tf), run_oracle(ev, W, H, p, tf), p["C"])


def test_checkpoint_and_resume_match_uninterrupted():
    rng = np.random.default_rng(15)
    W, H = 120, 80
    ev = random_events(rng, W, H, 100_000, 0, 2_000_000, hot=(3, 4, 0.02))
    p = P(render_decay=1, b=2.2)
    cut = 1_000_000
    tf1 = np.arange(100_000, cut + 1, 100_000)
    tf2 = np.arange(cut + 100_000, 2_000_001, 100_000)
    whole = run_gpu(ev, W, H, p, np.concatenate([tf1, tf2]), tuning=EXACT)
    first, second = ev[ev["t"] <= cut], ev[ev["t"] > cut]
    with GpuStream(W, H, p, EXACT) as g:
        assert g.push(first) == 0
        rc, fa = g.render_frames(tf1)
        S, T = g.state()
    with GpuStream(W, H, p, EXACT) as g:
        assert g.set_state(S, T) == 0
        assert g.push(second) == 0
        rc, fb = g.render_frames(tf2)
        S2, T2 = g.state()
    assert np.array_equal(S2, whole["S"]) and np.array_equal(T2, whole["T"])
    assert np.array_equal(np.concatenate([fa, fb]), whole["frames"])


def test_set_state_validation_and_decay_view_of_restored_state():
    rng = np.random.default_rng(16)
    W, H = 40, 20
    S0 = rng.uniform(-1, 1, W * H).astype(np.float32)
    T0 = rng.integers(0, 50_000, W * H).astype(np.int64)
    p = P(render_decay=1, b=1.3)
    with GpuStream(W, H, p) as g:
        assert g.set_state(S0, T0) == 0
        rc, fr = g.render_frames([60_000, 90_000, 160_000])
        assert rc == 0
        early = random_events(rng, W, H, 1, 0, 1)
        early["t"] = 10
        assert g.push(early) == g.esi.ESI_ETIMEORDER
    st = oracle.OracleState(W, H, oracle.OracleParams(**{k: p[k] for k in BASE}, render_decay=1))
    st.S[:] = S0.astype(np.float64)
    st.T[:] = T0
    for i, t in enumerate([60_000, 90_000, 160_000]):
        d = np.abs(fr[i].astype(int) - st.render(t).astype(int))
        assert d.max() <= 1


def test_device_push_and_device_output_match_host():
    rng = np.random.default_rng(17)
    W, H = 150, 100
    ev = random_events(rng, W, H, 40_000, 0, 1_000_000)
    p = P(render_decay=1)
    tf = np.arange(25_000, 1_000_001, 25_000)
    a = run_gpu(ev, W, H, p, tf)
    b = run_gpu(ev, W, H, p, tf, on_device=True)
    for k in ("S", "T", "frames"):
        assert np.array_equal(a[k], b[k]), k


def test_eq2_plain_integration_exact_with_k_zero():
    # k = 0 and non-binding bounds: S = C (n_plus - n_minus), exact for C = 0.25
    rng = np.random.default_rng(18)
    W, H = 70, 45
    ev = random_events(rng, W, H, 50_000, 0, 1_000_000)
    p = P(C=0.25, k_per_s=0.0, s_min=-1e6, s_max=1e6)
    g = run_gpu(ev, W, H, p, [1_000_000])
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    net = np.bincount(pix, weights=np.where(ev["p"] > 0, 1, -1), minlength=W * H)
    assert np.array_equal(g["S"].astype(np.float64), 0.25 * net)


def test_clamp_free_alg1_matches_oracle():
    rng = np.random.default_rng(19)
    W, H = 90, 60
    ev = random_events(rng, W, H, 60_000, 0, 1_000_000)
    p = P(k_per_s=5.0, b=2.7, s_min=-1e30, s_max=1e30)
    tf = [500_000, 1_000_000]
    compare(run_gpu(ev, W, H, p, tf), run_oracle(ev, W, H, p, tf), p["C"])


def test_launch_shapes_bit_identical_on_an_odd_width():
    # odd width: no row starts aligned, every width takes the per-pixel path
    rng = np.random.default_rng(41)
    W, H = 201, 77
    ev = random_events(rng, W, H, 40_000, 0, 400_000, hot=(200, 76, 0.05))
    p = P(render_decay=1)
    tf = np.arange(10_000, 400_001, 10_000)
    ref = run_gpu(ev, W, H, p, tf, tuning=EXACT)
    compare(ref, run_oracle(ev, W, H, p, tf), p["C"])
    for t in (dict(tile_w=64, tile_h=8), dict(tile_w=64, tile_h=4), dict(tile_w=32, tile_h=16),
              dict(tile_w=128, tile_h=16)):
        g = run_gpu(ev, W, H, p, tf, tuning={**t, **EXACT})
        assert np.array_equal(g["S"], ref["S"]), t
        assert np.array_equal(g["T"], ref["T"]), t
        assert np.array_equal(g["frames"], ref["frames"]), t


def test_large_pushes_are_checked_on_the_device():
    # pushes above 65536 events are checked chunk by chunk (2^21 events) on the
    # device: violations inside a chunk, across a chunk boundary and against
    # the previous push reject the whole push; a valid one goes through
    rng = np.random.default_rng(14)
    W, H = 64, 48
    n = (1 << 21) + 300_000
    ev = random_events(rng, W, H, n, 1_000, 60_000_000)
    p = P(render_decay=1)
    with GpuStream(W, H, p) as g:
        import torch

        def pinned(a):
            # page-locked host copy
            t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
            t.numpy()[:] = a.view(np.uint8)
            return t

        for where in (70_000, (1 << 21), (1 << 21) - 1, n - 1):
            bad = ev.copy()
            bad["t"][where] = bad["t"][where - 1] - 1
            assert g.push(bad) == g.esi.ESI_ETIMEORDER, where
            assert g.push(bad, on_device=True) == g.esi.ESI_ETIMEORDER, where
            assert g.esi.esi_push_events(g.h, pinned(bad), n, 0) == g.esi.ESI_ETIMEORDER, where
            assert g.stats().events_pushed == 0
        half = n // 2
        assert g.push(ev[:half]) == 0
        back = ev[half:].copy()
        back["t"][0] = ev["t"][half - 1] - 1          # earlier than the last pushed
        assert g.push(back) == g.esi.ESI_ETIMEORDER
        assert g.esi.esi_push_events(g.h, pinned(back), len(back), 0) == g.esi.ESI_ETIMEORDER
        third = half + (n - half) // 2
        assert g.esi.esi_push_events(g.h, pinned(ev[half:third]), third - half, 0) == 0
        assert g.push(ev[third:], on_device=True) == 0
        tf = np.arange(1_000_000, 60_000_001, 1_000_000)
        rc, fr = g.render_frames(tf)
        assert rc == 0
        S, T = g.state()
    ref = run_oracle(ev, W, H, p, tf)
    compare({"S": S, "T": T, "frames": fr}, ref, p["C"], "large pushes")


@pytest.mark.parametrize("small_first", [False, True])
def test_async_host_output_with_overlapping_pushes(small_first):
    # out_on_device = 2 returns once the render is queued; the next host push
    # runs on its own stream and may only overwrite ring slots the previous
    # render has binned.  Each push here fills the whole initial ring (2^20
    # events) and each render consumes all of it, so every push would
    # overwrite exactly the slots the previous render reads: the handle grows
    # the ring once instead of waiting.  After a small push (checked on the
    # host, whose time mirror the ring would have to carry) it waits instead.
    import torch
    rng = np.random.default_rng(15)
    W, H = 160, 120
    n = 1 << 20
    K = 4
    ev = random_events(rng, W, H, n * K, 0, 40_000_000, hot=(7, 9, 0.02))
    p = P(render_decay=1)
    per = 10
    tfs = [np.linspace(ev["t"][k * n] + 1, ev["t"][(k + 1) * n - 1], per).astype(np.int64)
           for k in range(K)]
    for k in range(K - 1):   # a frame at the push's last event time takes all of it
        assert ev["t"][(k + 1) * n] > tfs[k][-1]
    with GpuStream(W, H, p) as g:
        outs = []
        for k in range(K):
            if small_first and k == 0:
                assert g.push(ev[:1000]) == 0
                assert g.push(ev[1000:n]) == 0
            else:
                assert g.push(ev[k * n:(k + 1) * n]) == 0
            if k % 2 == 0:
                o = torch.empty((per, H, W), dtype=torch.uint8, pin_memory=True)
            else:
                o = np.empty((per, H, W), dtype=np.uint8)     # staged through the device
            assert g.esi.esi_render_frames(g.h, tfs[k], per, o, 2) == 0
            outs.append(o)
        assert g.esi.esi_synchronize(g.h) == 0
        frames = np.concatenate([o.numpy() if hasattr(o, "numpy") else o for o in outs])
        S, T = g.state()
        rc, st = g.esi.esi_get_stats(g.h)
        assert rc == 0 and st.ring_capacity >= n and st.ring_capacity & (st.ring_capacity - 1) == 0
        if small_first:   # the host time mirror keeps the ring at its size: pushes wait
            assert st.ring_grows == 0 and st.ring_capacity == n
    ref = run_oracle(ev, W, H, p, np.concatenate(tfs))
    compare({"S": S, "T": T, "frames": frames}, ref, p["C"], "async host output")


@pytest.mark.parametrize("W,H", [(1, 1), (1, 300), (300, 1), (65535, 2), (3, 65535), (4000, 3000)])
def test_extreme_sensor_shapes(W, H):
    # single pixels, single rows and columns, the widest and tallest sizes,
    # and a 12 M-pixel sensor (taller tiles and smaller chunks by default)
    rng = np.random.default_rng(W * 7 + H)
    n = min(200_000, max(50, W * H * 2))
    ev = random_events(rng, W, H, n, 0, 300_000, hot=(W - 1, H - 1, 0.05))
    p = P(render_decay=1)
    tf = np.array([100_000, 200_000, 300_000], dtype=np.int64)
    compare(run_gpu(ev, W, H, p, tf), run_oracle(ev, W, H, p, tf), p["C"], f"{W}x{H}")
