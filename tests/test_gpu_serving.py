"""Batched serving (esi_server_*) against the oracle and the single-sensor path.

Each stream of a server must give, frame for frame, what the oracle gives
for that stream alone (parity tolerance of esi_harness), and exactly what it
gives when served alone: streams never interact.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from esi_harness import (EXACT, STATE_TOL, GpuStream, compare, oracle_params, random_events,
                         run_oracle, state_error)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def _esi():
    from paper_2508_02238_gb300 import esi
    return esi


STREAMS = [
    # (W, H, params, generator)
    (64, 48, dict(C=0.25, k_per_s=20.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1), "random"),
    (346, 260, dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1), "sinusoid"),
    (200, 150, dict(C=0.15, k_per_s=5.0, b=1.5, s_min=-0.8, s_max=1.2, render_decay=0,
                    t_origin_us=3000), "random"),
    (130, 70, dict(C=0.3, k_per_s=0.0, b=2.0, s_min=-2.0, s_max=2.0, render_decay=1,
                   t_origin_us=7000), "random"),
    # Alg. 1 (no clamp) and Eq. 3 with exponential decay
    (96, 64, dict(C=0.2, k_per_s=30.0, b=2.0, s_min=-0.4, s_max=0.4, render_decay=1,
                  method=1), "random"),
    (120, 80, dict(C=0.2, k_per_s=50.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1,
                   method=2, t_origin_us=2000), "random"),
]


def make_stream_events(i, W, H, p, kind, t_end):
    t0 = p.get("t_origin_us", 0)
    if kind == "sinusoid":
        sc = synth.serving_stream(i, 2.0e6, (t_end - t0) / 1e6, W=W, H=H, t0_us=t0)
        return synth.generate(sc)
    rng = np.random.default_rng(100 + i)
    return random_events(rng, W, H, int(0.5 * W * H * (t_end - t0) / 1e5), t0, t_end,
                         hot=(W // 3, H // 2, 0.02))


def drive(esi, srv, ids, events, dims, t_end, tick_us=1000, start=0, on_tick=None):
    """Push 1 ms packets, tick every ms, read every finished frame."""
    frames = {sid: {} for sid in ids}
    pos = {sid: 0 for sid in ids}
    outs = {}
    for now in range(start + tick_us, t_end + 1, tick_us):
        for sid in ids:
            ev = events[sid]
            j = int(np.searchsorted(ev["t"], now, side="right"))
            if j > pos[sid]:
                pkt = np.ascontiguousarray(ev[pos[sid]:j])
                assert esi.esi_stream_push(srv, sid, pkt, len(pkt)) == 0
                pos[sid] = j
        if on_tick is not None:
            on_tick(now)
        assert esi.esi_server_tick(srv, now) == 0
        assert esi.esi_server_sync(srv) == 0
        for sid in ids:
            W, H = dims[sid]
            out = outs.setdefault(sid, np.empty((H, W), dtype=np.uint8))
            rc, tf, lat = esi.esi_stream_frame(srv, sid, out)
            if rc == 0:
                frames[sid][tf] = out.copy()
    return frames


def serve(stream_specs, t_end, use_graph=1, budget=256 << 20, tile_hs=None, retile=None,
          scan_chain=0, apply_mode=0, fuse_tick=0):
    """tile_hs: {spec index: tile height} set at open; retile: (time, {index: tile height})
    applied before that tick; scan_chain: the server's segmented-scan knob (33: off);
    apply_mode: when the server applies a stream's events (0: default); fuse_tick: one
    launch per tick where the streams allow it (0, 1) or always separate launches (2)."""
    esi = _esi()
    opts = esi.esi_server_opts()
    opts.use_graph = use_graph
    opts.scan_chain = scan_chain
    opts.apply_mode = apply_mode
    opts.fuse_tick = fuse_tick
    opts.host_pool_bytes = 64 << 20
    rc, srv = esi.esi_server_create(budget, opts, 0)
    assert rc == 0
    try:
        ids, events, specs, dims = [], {}, {}, {}
        for i, (W, H, p, kind) in stream_specs:
            rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**{**dict(t_origin_us=0), **p}))
            assert rc == 0
            ids.append(sid)
            events[sid] = make_stream_events(i, W, H, p, kind, t_end)
            dims[sid] = (W, H)
            specs[sid] = (i, W, H, p)
            if tile_hs and i in tile_hs:
                assert esi.esi_stream_set_tile_h(srv, sid, tile_hs[i]) == 0
        on_tick = None
        if retile is not None:
            def on_tick(now):
                if now == retile[0]:
                    for sid in ids:
                        th = retile[1].get(specs[sid][0])
                        if th:
                            assert esi.esi_stream_set_tile_h(srv, sid, th) == 0
        frames = drive(esi, srv, ids, events, dims, t_end, on_tick=on_tick)
        states = {}
        for sid in ids:
            W, H = dims[sid]
            S = np.empty(W * H, dtype=np.float32)
            T = np.empty(W * H, dtype=np.int64)
            assert esi.esi_stream_state(srv, sid, S, T) == 0
            states[sid] = (S, T)
        rc, st = esi.esi_server_get_stats(srv)
        assert rc == 0
        return {specs[sid][0]: (frames[sid], states[sid], events[sid]) for sid in ids}, st
    finally:
        esi.esi_server_destroy(srv)


def test_served_streams_match_the_oracle():
    t_end = 120_000
    res, st = serve(list(enumerate(STREAMS)), t_end)
    assert st.frames > 0 and st.kernel_launches_per_tick >= 2
    for i, (W, H, p, kind) in enumerate(STREAMS):
        frames, (S, T), ev = res[i]
        t0 = p.get("t_origin_us", 0)
        expect_tf = list(range(t0 + 10_000, t_end + 1, 10_000))
        assert sorted(frames) == expect_tf, (i, sorted(frames)[:3])
        pp = {**dict(t_origin_us=0), **p}
        used = ev[ev["t"] <= t_end]
        # frames at their times; the state holds every event the server has
        # seen by the last tick (events after a stream's last frame included)
        st_ref = oracle.OracleState(W, H, oracle_params(pp))
        ref_frames, n_used = st_ref.replay(used, expect_tf)
        st_ref.integrate(used[n_used:])
        got = {"S": S, "T": T, "frames": np.stack([frames[t] for t in expect_tf])}
        compare(got, {"S": st_ref.S, "T": st_ref.T, "frames": ref_frames}, pp["C"], f"stream {i}")


def test_both_apply_modes_match_each_other():
    # events applied every tick or only in frame ticks: the same frames and
    # states (with the scan off, bit for bit; the record groups differ)
    esi = _esi()
    t_end = 90_000
    specs = list(enumerate(STREAMS[:4]))
    every, st_e = serve(specs, t_end, scan_chain=33, apply_mode=esi.ESI_APPLY_EVERY_TICK)
    frames_only, st_f = serve(specs, t_end, scan_chain=33, apply_mode=esi.ESI_APPLY_AT_FRAMES)
    for i, _ in specs:
        fe, (Se, Te), _ = every[i]
        ff, (Sf, Tf), _ = frames_only[i]
        assert sorted(fe) == sorted(ff)
        for t in fe:
            assert np.array_equal(fe[t], ff[t]), (i, t)
        assert np.array_equal(Se, Sf) and np.array_equal(Te, Tf)
    assert st_e.frames == st_f.frames and st_e.events == st_f.events


def test_frame_only_mode_holds_events_back_until_a_frame_or_a_state_read():
    esi = _esi()
    W, H = 96, 40
    opts = esi.esi_server_opts()
    opts.apply_mode = esi.ESI_APPLY_AT_FRAMES
    opts.host_pool_bytes = 16 << 20
    rc, srv = esi.esi_server_create(64 << 20, opts, 0)
    assert rc == 0
    try:
        pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        ev = random_events(np.random.default_rng(3), W, H, 3000, 0, 4000)
        assert esi.esi_stream_push(srv, sid, ev, len(ev)) == 0
        for now in (1000, 2000, 4000):
            assert esi.esi_server_tick(srv, now) == 0
        assert esi.esi_server_sync(srv) == 0
        rc, st = esi.esi_server_get_stats(srv)
        assert rc == 0 and st.events == 0 and st.frames == 0   # no frame due before 10 ms
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, sid, S, T) == 0       # applies the held events
        rc, st = esi.esi_server_get_stats(srv)
        assert st.events == len(ev)
        ref = oracle.OracleState(W, H, oracle_params(pp))
        ref.integrate(ev)
        assert np.array_equal(T, ref.T)
        assert state_error(S, ref.S, pp["C"]) <= STATE_TOL
    finally:
        esi.esi_server_destroy(srv)


def test_event_rings_grow_and_refuse_pushes_beyond_the_host_pool():
    # a stream's ring starts at 16384 events and grows on demand inside the
    # pinned host pool (to a power of two with a quarter to spare); a push
    # that cannot fit is refused whole
    # (ESI_ENOMEM, with the reason in esi_server_last_error) and the stream
    # carries on with the events it had
    esi = _esi()
    W, H = 200, 150
    opts = esi.esi_server_opts()
    opts.host_pool_bytes = 8 << 20            # 524288 events
    rc, srv = esi.esi_server_create(64 << 20, opts, 0)
    assert rc == 0
    try:
        pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        ev = random_events(np.random.default_rng(11), W, H, 400_000, 0, 40_000)
        a, b = 100_000, 300_000
        assert esi.esi_stream_push(srv, sid, ev[:a], a) == 0      # grows to 131072 events
        assert esi.esi_stream_push(srv, sid, ev[a:b], b - a) == esi.ESI_ENOMEM
        assert "host pool full" in esi.esi_server_last_error(srv)
        t_a = int(ev["t"][a - 1])                                  # about 10 ms
        for now in list(range(1000, t_a, 1000)) + [t_a]:
            assert esi.esi_server_tick(srv, now) == 0
        assert esi.esi_server_sync(srv) == 0
        # the refused push left nothing behind: the rest goes in packet by packet
        for lo in range(a, len(ev), 20_000):
            part = ev[lo:lo + 20_000]
            assert esi.esi_stream_push(srv, sid, part, len(part)) == 0
            assert esi.esi_server_tick(srv, int(part["t"][-1])) == 0
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, sid, S, T) == 0
        ref = oracle.OracleState(W, H, oracle_params(pp))
        ref.integrate(ev)
        assert np.array_equal(T, ref.T)
        assert state_error(S, ref.S, pp["C"]) <= STATE_TOL
        rc, n_done = esi.esi_stream_frames_done(srv, sid)
        assert rc == 0 and n_done == int(ev["t"][-1]) // 10_000    # 10, 20, 30 ms
        rc, st = esi.esi_server_get_stats(srv)
        assert st.ring_grows >= 1 and st.host_pool_peak_bytes >= (131072 * 16)
    finally:
        esi.esi_server_destroy(srv)


def test_a_ring_grown_for_a_burst_shrinks_once_applied():
    esi = _esi()
    W, H = 120, 90
    opts = esi.esi_server_opts()
    opts.host_pool_bytes = 64 << 20
    rc, srv = esi.esi_server_create(64 << 20, opts, 0)
    assert rc == 0
    try:
        pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        ev = random_events(np.random.default_rng(21), W, H, 600_000, 0, 25_000)
        burst = int(np.searchsorted(ev["t"], 5000, side="right"))   # 120 k events
        assert esi.esi_stream_push(srv, sid, ev[:burst], burst) == 0
        assert esi.esi_server_tick(srv, 5000) == 0
        assert esi.esi_server_sync(srv) == 0
        rc, st = esi.esi_server_get_stats(srv)
        big = st.host_pool_peak_bytes
        assert st.ring_grows == 1 and big >= 262144 * 16
        lo = burst
        for now in range(6000, 25_001, 1000):                        # 24 k events per ms
            hi = int(np.searchsorted(ev["t"], now, side="right"))
            assert esi.esi_stream_push(srv, sid, ev[lo:hi], hi - lo) == 0
            assert esi.esi_server_tick(srv, now) == 0
            lo = hi
        assert esi.esi_server_sync(srv) == 0
        rc, st = esi.esi_server_get_stats(srv)
        assert st.host_pool_used_bytes < 262144 * 16                 # back to a small ring
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, sid, S, T) == 0
        ref = oracle.OracleState(W, H, oracle_params(pp))
        ref.integrate(ev[:lo])
        assert np.array_equal(T, ref.T)
        assert state_error(S, ref.S, pp["C"]) <= STATE_TOL
    finally:
        esi.esi_server_destroy(srv)


def test_tick_trace_records_every_tick_with_work():
    esi = _esi()
    W, H = 96, 40
    rc, srv = esi.esi_server_create(64 << 20, None, 0)
    assert rc == 0
    try:
        pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        ev = random_events(np.random.default_rng(5), W, H, 20_000, 0, 30_000)
        n_ticks, lo = 0, 0
        for now in range(1000, 30_001, 1000):
            hi = int(np.searchsorted(ev["t"], now, side="right"))
            part = ev[lo:hi]
            lo = hi
            assert esi.esi_stream_push(srv, sid, part, len(part)) == 0
            assert esi.esi_server_tick(srv, now) == 0
            n_ticks += 1
        assert esi.esi_server_sync(srv) == 0
        rc, tr = esi.esi_server_trace(srv)
        assert rc == 0 and len(tr) == n_ticks
        assert int(tr["events"].sum()) == len(ev)
        assert int(tr["frames"].sum()) == 3
        assert np.all(np.diff(tr["call_ns"]) > 0)
        # a small tick can finish on the device before its call has returned
        assert np.all(tr["issued_ns"] >= tr["call_ns"]) and np.all(tr["ready_ns"] >= tr["call_ns"])
        assert np.all(tr["kernels_ms"] > 0) and tr["gap_ms"][0] == -1.0
        assert esi.esi_server_reset_stats(srv) == 0
        rc, tr = esi.esi_server_trace(srv)
        assert rc == 0 and len(tr) == 0
    finally:
        esi.esi_server_destroy(srv)


def test_close_with_frames_in_flight_and_an_id_reused_at_once():
    # esi_stream_close returns without waiting: the closed stream's frames
    # still reach its sink, and a stream opened on the same id right away
    # sees none of them
    esi = _esi()
    W, H = 120, 90
    pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
    rc, srv = esi.esi_server_create(64 << 20, None, 0)
    assert rc == 0
    try:
        rc, a = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        sink = np.zeros((3, H, W), dtype=np.uint8)
        sink_t = np.zeros(3, dtype=np.int64)
        assert esi.esi_stream_set_frame_sink(srv, a, sink, 3, sink_t) == 0
        ev_a = random_events(np.random.default_rng(31), W, H, 60_000, 0, 30_000)
        assert esi.esi_stream_push(srv, a, ev_a, len(ev_a)) == 0
        assert esi.esi_server_tick(srv, 30_000) == 0          # frames 10, 20, 30 ms queued
        assert esi.esi_stream_close(srv, a) == 0               # no wait
        pb = dict(pp, C=0.3, t_origin_us=30_000)
        rc, b = esi.esi_stream_open(srv, W, H, esi.make_params(**pb))
        assert rc == 0 and b == a                              # the id comes back at once
        ev_b = random_events(np.random.default_rng(32), W, H, 20_000, 30_000, 50_000)
        assert esi.esi_stream_push(srv, b, ev_b, len(ev_b)) == 0
        assert esi.esi_server_tick(srv, 45_000) == 0           # frame 40 ms of the new stream
        assert esi.esi_server_sync(srv) == 0
        rc, n_b = esi.esi_stream_frames_done(srv, b)
        assert rc == 0 and n_b == 1
        out = np.empty((H, W), dtype=np.uint8)
        rc, tf = esi.esi_stream_frame_seq(srv, b, 0, out)
        assert rc == 0 and tf == 40_000
        ref_b = oracle.OracleState(W, H, oracle_params(pb))
        fb, _ = ref_b.replay(ev_b, np.array([40_000], dtype=np.int64))
        assert int(np.abs(out.astype(np.int16) - fb[0].astype(np.int16)).max()) <= 1
        ref_a = oracle.OracleState(W, H, oracle_params(pp))
        fa, _ = ref_a.replay(ev_a, np.array([10_000, 20_000, 30_000], dtype=np.int64))
        assert list(sink_t) == [10_000, 20_000, 30_000]
        assert int(np.abs(sink.astype(np.int16) - fa.astype(np.int16)).max()) <= 1
    finally:
        esi.esi_server_destroy(srv)


def test_served_events_outside_the_sensor_are_dropped_and_counted():
    esi = _esi()
    W, H = 100, 60
    pp = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1, t_origin_us=0)
    rc, srv = esi.esi_server_create(64 << 20, None, 0)
    assert rc == 0
    try:
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**pp))
        assert rc == 0
        ev = random_events(np.random.default_rng(41), W + 7, H + 3, 30_000, 0, 20_000)
        bad = int(np.count_nonzero((ev["x"] >= W) | (ev["y"] >= H)))
        assert bad > 0
        assert esi.esi_stream_push(srv, sid, ev, len(ev)) == 0
        assert esi.esi_server_tick(srv, 20_000) == 0
        assert esi.esi_server_sync(srv) == 0
        rc, st = esi.esi_server_get_stats(srv)
        assert rc == 0 and st.events_dropped == bad and st.events == len(ev)
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, sid, S, T) == 0
        ref = oracle.OracleState(W, H, oracle_params(pp))
        ref.integrate(ev)
        assert np.array_equal(T, ref.T)
        assert state_error(S, ref.S, pp["C"]) <= STATE_TOL
        out = np.empty((H, W), dtype=np.uint8)
        rc, tf = esi.esi_stream_frame_seq(srv, sid, 1, out)
        assert rc == 0 and tf == 20_000
    finally:
        esi.esi_server_destroy(srv)


def test_apply_mode_validation():
    esi = _esi()
    for mode, threads, ok in ((0, 0, True), (1, 1, True), (2, 16, True), (3, 0, False),
                              (-1, 0, False), (0, 17, False)):
        opts = esi.esi_server_opts()
        opts.apply_mode, opts.copy_threads, opts.fuse_tick = mode, threads, mode % 3
        rc, srv = esi.esi_server_create(1 << 20, opts, 0)
        assert (rc == 0) == ok, (mode, threads, rc)
        if rc == 0:
            esi.esi_server_destroy(srv)


def test_each_stream_is_the_same_alone_and_in_the_mix():
    t_end = 80_000
    mix, _ = serve(list(enumerate(STREAMS)), t_end)
    for i, spec in enumerate(STREAMS):
        alone, _ = serve([(i, spec)], t_end)
        fa, (Sa, Ta), _ = alone[i]
        fm, (Sm, Tm), _ = mix[i]
        assert sorted(fa) == sorted(fm)
        for t in fa:
            assert np.array_equal(fa[t], fm[t]), (i, t)
        assert np.array_equal(Sa, Sm) and np.array_equal(Ta, Tm)


def test_served_stream_equals_single_sensor_handle():
    # the server and esi_render_frames run the same kernels on the same events
    # (with the scan off on both: ticks and one render group records apart)
    W, H, p, kind = STREAMS[1]
    t_end = 100_000
    res, _ = serve([(1, STREAMS[1])], t_end, scan_chain=33)
    frames, (S, T), ev = res[1]
    tf = sorted(frames)
    used = ev[ev["t"] <= t_end]
    with GpuStream(W, H, {**dict(t_origin_us=0), **p}, EXACT) as g:
        assert g.push(used) == 0
        rc, fr = g.render_frames(tf)
        assert rc == 0
        rc, _ = g.render_frame(t_end)   # the server has applied everything up to t_end
        assert rc == 0
        Sh, Th = g.state()
    assert np.array_equal(np.stack([frames[t] for t in tf]), fr)
    assert np.array_equal(S, Sh) and np.array_equal(T, Th)


def test_fused_tick_launch_equals_separate_launches():
    # streams that all use 8-row tiles and share render mode and decay kind
    # (row widths with and without 4-pixel alignment): one persistent launch
    # per tick gives exactly what the binning launch plus per-variant tile
    # launches give, graph or not
    specs = [(1, STREAMS[1]), (2, (200, 150, dict(STREAMS[1][2]), "random")),
             (0, (64, 48, dict(STREAMS[1][2]), "random")), (5, (131, 77, dict(STREAMS[1][2]), "random"))]
    t_end = 70_000
    sep, st_s = serve(specs, t_end, fuse_tick=2)
    fus, st_f = serve(specs, t_end, fuse_tick=1)
    fus_direct, st_d = serve(specs, t_end, fuse_tick=1, use_graph=0)
    assert st_f.kernel_launches_per_tick == 1 and st_d.kernel_launches_per_tick == 1
    assert st_s.kernel_launches_per_tick >= 3
    for i, _ in specs:
        for other in (fus, fus_direct):
            assert sorted(sep[i][0]) == sorted(other[i][0])
            for t in sep[i][0]:
                assert np.array_equal(sep[i][0][t], other[i][0][t]), (i, t)
            assert np.array_equal(sep[i][1][0], other[i][1][0]) and np.array_equal(sep[i][1][1], other[i][1][1])


def test_fused_tick_is_skipped_when_streams_differ_in_tile_height():
    specs = list(enumerate(STREAMS[:2]))
    res, st = serve(specs, 40_000, tile_hs={0: 4})
    assert st.kernel_launches_per_tick >= 3
    ref, _ = serve(specs, 40_000, fuse_tick=2, tile_hs={0: 4})
    for i, _ in specs:
        for t in ref[i][0]:
            assert np.array_equal(ref[i][0][t], res[i][0][t])


def test_graph_and_direct_launches_agree():
    t_end = 60_000
    a, _ = serve(list(enumerate(STREAMS[:3])), t_end, use_graph=1)
    b, _ = serve(list(enumerate(STREAMS[:3])), t_end, use_graph=0)
    for i in range(3):
        for t in a[i][0]:
            assert np.array_equal(a[i][0][t], b[i][0][t])
        assert np.array_equal(a[i][1][0], b[i][1][0])


def test_admission_by_state_memory_and_join_leave():
    esi = _esi()
    W, H = 346, 260
    per_stream = 12 * W * H + 4096
    rc, srv = esi.esi_server_create(3 * per_stream, None, 0)
    assert rc == 0
    try:
        p = esi.make_params(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
        ids = []
        for _ in range(3):
            rc, sid = esi.esi_stream_open(srv, W, H, p)
            assert rc == 0
            ids.append(sid)
        rc, _ = esi.esi_stream_open(srv, W, H, p)
        assert rc == esi.ESI_EBUSY                     # the budget is full
        rc, st = esi.esi_server_get_stats(srv)
        assert st.streams_open == 3 and st.state_bytes_used <= st.state_budget_bytes
        # run a little, then one stream leaves and a new one is admitted
        rng = np.random.default_rng(5)
        evs = {sid: random_events(rng, W, H, 20_000, 0, 50_000) for sid in ids}
        pos = {sid: 0 for sid in ids}
        for now in range(1000, 30_001, 1000):
            for sid in ids:
                e = evs[sid]
                j = int(np.searchsorted(e["t"], now, side="right"))
                pkt = np.ascontiguousarray(e[pos[sid]:j])
                pos[sid] = j
                assert esi.esi_stream_push(srv, sid, pkt, len(pkt)) == 0
            assert esi.esi_server_tick(srv, now) == 0
        assert esi.esi_stream_close(srv, ids[1]) == 0
        rc, new = esi.esi_stream_open(srv, W, H, p)
        assert rc == 0
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, new, S, T) == 0
        assert np.all(S == 0) and np.all(T == 0)       # Alg. 2 initial state
        out = np.empty((H, W), dtype=np.uint8)
        assert esi.esi_stream_frame(srv, new, out)[0] == esi.ESI_ESTATE
        rc, tf, _ = esi.esi_stream_frame(srv, ids[0], out)
        assert rc == 0 and tf == 30_000
        # the survivor matches the oracle over the same events
        e0 = evs[ids[0]]
        used = e0[e0["t"] <= 30_000]
        assert esi.esi_stream_state(srv, ids[0], S, T) == 0
        ref = oracle.OracleState(W, H, oracle_params(dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0,
                                                          s_max=1.0, render_decay=1)))
        ref.integrate(used)
        compare({"S": S, "T": T}, {"S": ref.S, "T": ref.T}, 0.2, "survivor")
    finally:
        esi.esi_server_destroy(srv)


def test_push_validation():
    esi = _esi()
    rc, srv = esi.esi_server_create(64 << 20, None, 0)
    assert rc == 0
    try:
        p = esi.make_params(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)
        rc, sid = esi.esi_stream_open(srv, 32, 32, p)
        assert rc == 0
        ev = random_events(np.random.default_rng(1), 32, 32, 10, 0, 1000)
        bad = ev.copy()
        bad["t"][3] = bad["t"][2] - 1
        assert esi.esi_stream_push(srv, sid, bad, len(bad)) == esi.ESI_ETIMEORDER
        assert esi.esi_stream_push(srv, sid, ev, len(ev)) == 0
        assert esi.esi_stream_push(srv, 99, ev, len(ev)) == esi.ESI_EINVAL
        rc, _ = esi.esi_stream_open(srv, 5000, 5000, p)
        assert rc == esi.ESI_ERANGE
    finally:
        esi.esi_server_destroy(srv)


def test_per_stream_tile_heights_are_bit_identical():
    # tiles only organise the work: every pixel applies its events in the same
    # order with the same arithmetic at any tile height (scan off), and the
    # height may change between ticks
    t_end = 60_000
    specs = list(enumerate(STREAMS))
    base, _ = serve(specs, t_end, scan_chain=33)
    mixed, st = serve(specs, t_end, tile_hs={0: 4, 1: 16, 2: 4, 3: 16}, scan_chain=33)
    moved, _ = serve(specs, t_end, tile_hs={1: 4}, retile=(25_000, {0: 16, 1: 8, 2: 16, 3: 4}),
                     scan_chain=33)
    for other in (mixed, moved):
        for i in range(len(STREAMS)):
            fa, (Sa, Ta), _ = base[i]
            fb, (Sb, Tb), _ = other[i]
            assert sorted(fa) == sorted(fb)
            for t in fa:
                assert np.array_equal(fa[t], fb[t]), (i, t)
            assert np.array_equal(Sa, Sb) and np.array_equal(Ta, Tb)
    assert st.kernel_launches_per_tick >= 2


def test_stream_tile_height_validation_and_autotune():
    esi = _esi()
    rc, srv = esi.esi_server_create(64 << 20, None, 0)
    assert rc == 0
    try:
        W, H, p, kind = STREAMS[1]
        rc, sid = esi.esi_stream_open(srv, W, H, esi.make_params(**{**dict(t_origin_us=0), **p}))
        assert rc == 0
        for bad in (0, 2, 12, 32):
            assert esi.esi_stream_set_tile_h(srv, sid, bad) == esi.ESI_EINVAL
        assert esi.esi_stream_set_tile_h(srv, sid + 1, 8) == esi.ESI_EINVAL
        sample = make_stream_events(1, W, H, p, kind, 100_000)
        rc, th = esi.esi_stream_autotune(srv, sid, sample, len(sample), esi.ESI_AUTOTUNE_FORCE)
        assert rc == 0 and th in (4, 8, 16)
        rc, th2 = esi.esi_stream_autotune(srv, sid, sample, len(sample), 0)   # cached
        assert rc == 0 and th2 == th
        # the stream's state is untouched (Alg. 2 initial state)
        S = np.empty(W * H, dtype=np.float32)
        T = np.empty(W * H, dtype=np.int64)
        assert esi.esi_stream_state(srv, sid, S, T) == 0
        assert np.all(S == 0) and np.all(T == 0)
        # and the tuned stream still matches the oracle
        ev = sample[sample["t"] <= 50_000]
        frames = drive(esi, srv, [sid], {sid: ev}, {sid: (W, H)}, 50_000)
        assert esi.esi_stream_state(srv, sid, S, T) == 0
        tf = sorted(frames[sid])
        assert tf == list(range(10_000, 50_001, 10_000))
        pp = {**dict(t_origin_us=0), **p}
        ref = oracle.OracleState(W, H, oracle_params(pp))
        ref_frames, n_used = ref.replay(ev, tf)
        ref.integrate(ev[n_used:])
        compare({"S": S, "T": T, "frames": np.stack([frames[sid][t] for t in tf])},
                {"S": ref.S, "T": ref.T, "frames": ref_frames}, pp["C"], "autotuned stream")
    finally:
        esi.esi_server_destroy(srv)


def _state_bytes(W, H):
    P = W * H
    return ((P * 4 + 255) // 256 * 256 + P * 8 + 255) // 256 * 256


@pytest.mark.parametrize("realtime", [0, 1])
def test_executor_join_leave_and_admission(realtime):
    """Streams join and leave through the executor's OPEN / CLOSE packets; a
    join that does not fit the state budget is refused and its events dropped;
    a later join fits again once a stream has left.  As fast as possible, and
    paced by the wall clock (where a packet that makes a frame due is
    rendered before the packets behind it are taken)."""
    esi = _esi()
    P = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
    t_end = 60_000
    # slot: (W, H, join, leave, rate)
    plan = [(346, 260, 0, None, 1.5e6), (640, 480, 0, 30_000, 2.0e6),
            (346, 260, 10_000, None, 0.8e6), (640, 480, 20_000, None, 1.0e6),
            (640, 480, 40_000, None, 3.0e6)]
    budget = 2 * _state_bytes(346, 260) + _state_bytes(640, 480) + 4096
    evs, specs = [], []
    for k, (W, H, tj, tl, rate) in enumerate(plan):
        dur = ((tl or t_end) - tj) / 1e6
        if W == 346:
            sc = synth.serving_stream(k, rate, dur, t0_us=tj)
        else:
            sc = synth.blobs_640x480(duration_s=dur, seed=5000 + k, t0_us=tj)
            sc.keep_prob = rate / synth.BLOBS_NATURAL_RATE
        evs.append(synth.generate(sc))
        sp = esi.esi_stream_spec()
        sp.width, sp.height, sp.tile_h = W, H, (4, 8, 16, 8, 4)[k]
        sp.params = esi.make_params(**P, t_origin_us=tj)
        specs.append(sp)
    items = []
    for k, (W, H, tj, tl, rate) in enumerate(plan):
        items.append((tj, 0, k, ctypes.addressof(specs[k]), 0, esi.ESI_PACKET_OPEN))
        ev = evs[k]
        lo = 0
        for a in range(tj + 1000, (tl or t_end) + 1, 1000):
            hi = int(np.searchsorted(ev["t"], a, side="right"))
            items.append((a, 1, k, ev.ctypes.data + lo * 16, hi - lo, esi.ESI_PACKET_EVENTS))
            lo = hi
        if tl is not None:
            items.append((tl, 2, k, 0, 0, esi.ESI_PACKET_CLOSE))
    items.sort(key=lambda x: (x[0], x[1], x[2]))
    pk = (esi.esi_packet * len(items))()
    for j, (a, _, k, p_, n, kind) in enumerate(items):
        pk[j].stream, pk[j].kind, pk[j].arrival_us, pk[j].ev, pk[j].n = k, kind, a, p_, n
    rc, srv = esi.esi_server_create(budget, None, 0)
    assert rc == 0
    try:
        assert esi.esi_server_run(srv, pk, len(items), 1000, t_end, realtime) == 0
        rc, st = esi.esi_server_get_stats(srv)
        assert rc == 0
        assert st.streams_admitted == 4 and st.streams_refused == 1
        assert st.events_refused == len(evs[3])
        assert st.streams_open == 3
        assert [sp.stream_id >= 0 for sp in specs] == [True, False, True, False, True]
        # frames every 10 ms from each stream's join up to the end or its leave
        # (slot 1's 30 ms frame is rendered before it closes)
        assert st.frames == 6 + 3 + 5 + 2
        for k in (0, 2, 4):
            W, H, tj, tl, rate = plan[k]
            sid = specs[k].stream_id
            S = np.empty(W * H, dtype=np.float32)
            T = np.empty(W * H, dtype=np.int64)
            assert esi.esi_stream_state(srv, sid, S, T) == 0
            out = np.empty((H, W), dtype=np.uint8)
            rc, tf, _ = esi.esi_stream_frame(srv, sid, out)
            assert rc == 0 and tf == t_end
            ev = evs[k]
            ref = oracle.OracleState(W, H, oracle_params({**P, "t_origin_us": tj}))
            ref_frames, n_used = ref.replay(ev, [t_end])
            ref.integrate(ev[n_used:])
            compare({"S": S, "T": T, "frames": out[None]},
                    {"S": ref.S, "T": ref.T, "frames": ref_frames}, P["C"], f"slot {k}")
        # the executor rejects malformed control packets
        bad = (esi.esi_packet * 1)()
        bad[0].stream, bad[0].kind, bad[0].arrival_us = 0, 7, 0
        assert esi.esi_server_run(srv, bad, 1, 1000, 0, 0) == esi.ESI_EINVAL
        bad[0].kind, bad[0].ev = esi.ESI_PACKET_OPEN, None
        assert esi.esi_server_run(srv, bad, 1, 1000, 0, 0) == esi.ESI_EINVAL
        bad[0].kind, bad[0].stream = esi.ESI_PACKET_EVENTS, 1 << 20
        assert esi.esi_server_run(srv, bad, 1, 1000, 0, 0) == esi.ESI_EINVAL
    finally:
        esi.esi_server_destroy(srv)


def test_large_and_small_streams_in_one_tick():
    # a 1280x720 stream at tile height 4 has 1800 tiles: its binning job
    # finds same-tile lanes by ballots, while the small stream's job in the
    # same launch uses the shared-memory mask words
    big = (1280, 720, dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1),
           "random")
    small = STREAMS[0]
    t_end = 40_000
    res, _ = serve([(0, big), (1, small)], t_end, tile_hs={0: 4})
    for i, (W, H, p, kind) in ((0, big), (1, small)):
        frames, (S, T), ev = res[i]
        expect_tf = list(range(10_000, t_end + 1, 10_000))
        assert sorted(frames) == expect_tf
        pp = {**dict(t_origin_us=0), **p}
        used = ev[ev["t"] <= t_end]
        st_ref = oracle.OracleState(W, H, oracle_params(pp))
        ref_frames, n_used = st_ref.replay(used, expect_tf)
        st_ref.integrate(used[n_used:])
        got = {"S": S, "T": T, "frames": np.stack([frames[t] for t in expect_tf])}
        compare(got, {"S": st_ref.S, "T": st_ref.T, "frames": ref_frames}, pp["C"], f"stream {i}")
