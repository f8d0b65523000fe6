"""Batched serving at the size of the serving workloads, against the oracle.

The 64-stream workload (64 sinusoid form 346x260 streams, lognormal rates
0.2-5 Mev/s, Poisson packets with a 1 ms mean gap, 100 frames/s, 0.25 s: the
seeded workload the bench serves) and a mixed workload with all three sensor
sizes (1280x720 checkerboard, 640x480 blob and 346x260 sinusoid forms) whose
streams join and leave on a seeded schedule.  Packets are pushed as they
arrive, the server ticks every millisecond, and every finished frame is read
back by number.  Each stream's frames and final state must match what the
FP64 oracle gives for that stream alone (tolerances of esi_harness), and a
stream served alone must give bit for bit what it gives in the mix.
"""
import numpy as np
import pytest

import oracle
import synth
from esi_harness import compare, oracle_params

pytestmark = pytest.mark.gpu

PARAMS = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
FRAME_US = 10_000


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def serve_schedule(specs, t_end, budget=1 << 30, tick_us=1000):
    """specs: dicts with W, H, events, arrivals, t_join_us, t_leave_us (or
    None), tile_h.  Returns per spec: {t_frame: frame}, final (S, T) or None
    (left), and server stats."""
    from paper_2508_02238_gb300 import esi
    opts = esi.esi_server_opts()
    opts.max_streams = max(256, len(specs))
    rc, srv = esi.esi_server_create(budget, opts, 0)
    assert rc == 0
    n = len(specs)
    sid = [None] * n
    closed = [False] * n
    pos, ai, nread = [0] * n, [0] * n, [0] * n
    frames = [dict() for _ in range(n)]
    bufs = {}

    def read_frames(k):
        rc, done = esi.esi_stream_frames_done(srv, sid[k])
        assert rc == 0
        W, H = specs[k]["W"], specs[k]["H"]
        out = bufs.setdefault((W, H), np.empty((H, W), dtype=np.uint8))
        for seq in range(nread[k], done):
            rc, tf = esi.esi_stream_frame_seq(srv, sid[k], seq, out)
            assert rc == 0, (k, seq, esi.esi_strerror(rc))
            frames[k][tf] = out.copy()
        nread[k] = done

    def due(k, upto):
        sp = specs[k]
        return max(0, (upto - sp["t_join_us"]) // FRAME_US)

    try:
        for now in range(tick_us, t_end + tick_us, tick_us):
            for k, sp in enumerate(specs):
                if closed[k]:
                    continue
                if sid[k] is None:
                    if sp["t_join_us"] > now:
                        continue
                    prm = esi.make_params(**PARAMS, t_origin_us=sp["t_join_us"])
                    rc, sid[k] = esi.esi_stream_open(srv, sp["W"], sp["H"], prm)
                    assert rc == 0, esi.esi_strerror(rc)
                    assert esi.esi_stream_set_tile_h(srv, sid[k], sp.get("tile_h", 8)) == 0
                ev, arr = sp["events"], sp["arrivals"]
                while ai[k] < len(arr) and arr[ai[k]] <= now:
                    j = int(np.searchsorted(ev["t"], arr[ai[k]], side="right"))
                    if j > pos[k]:
                        pkt = np.ascontiguousarray(ev[pos[k]:j])
                        assert esi.esi_stream_push(srv, sid[k], pkt, len(pkt)) == 0
                        pos[k] = j
                    assert esi.esi_stream_watermark(srv, sid[k], int(arr[ai[k]])) == 0
                    ai[k] += 1
            assert esi.esi_server_tick(srv, now) == 0
            assert esi.esi_server_sync(srv) == 0
            for k, sp in enumerate(specs):
                if sid[k] is None or closed[k]:
                    continue
                read_frames(k)
                tl = sp["t_leave_us"]
                if tl is not None and tl <= now:
                    # render what is due up to the leave time, then close
                    for _ in range(16):
                        if nread[k] >= due(k, tl):
                            break
                        assert esi.esi_server_tick(srv, now) == 0
                        assert esi.esi_server_sync(srv) == 0
                        read_frames(k)
                    assert esi.esi_stream_close(srv, sid[k]) == 0
                    closed[k] = True
        # drain: every due frame of the streams still open
        for _ in range(16):
            pending = [k for k in range(n) if sid[k] is not None and not closed[k]
                       and nread[k] < due(k, t_end)]
            if not pending:
                break
            assert esi.esi_server_tick(srv, t_end) == 0
            assert esi.esi_server_sync(srv) == 0
            for k in pending:
                read_frames(k)
        states = []
        for k, sp in enumerate(specs):
            if sid[k] is None or closed[k]:
                states.append(None)
                continue
            S = np.empty(sp["W"] * sp["H"], dtype=np.float32)
            T = np.empty(sp["W"] * sp["H"], dtype=np.int64)
            assert esi.esi_stream_state(srv, sid[k], S, T) == 0
            states.append((S, T))
        rc, st = esi.esi_server_get_stats(srv)
        assert rc == 0
        return frames, states, st
    finally:
        esi.esi_server_destroy(srv)


def check_against_oracle(specs, frames, states, t_end):
    """Every stream's frames (and final state if it stayed) against the oracle
    run on that stream alone; returns the maxima over the streams."""
    worst = {"state_err": 0.0, "frame_max_lsb": 0, "frame_off_by_one": 0, "frames": 0}
    for k, sp in enumerate(specs):
        t0 = sp["t_join_us"]
        t1 = sp["t_leave_us"] if sp["t_leave_us"] is not None else t_end
        tf = np.arange(t0 + FRAME_US, t1 + 1, FRAME_US, dtype=np.int64)
        assert sorted(frames[k]) == tf.tolist(), (k, sorted(frames[k])[:3], tf[:3])
        ev = sp["events"]
        p = dict(PARAMS, t_origin_us=t0)
        ref = oracle.OracleState(sp["W"], sp["H"], oracle_params(p))
        ref_frames, used = ref.replay(ev, tf)
        got = {"frames": np.stack([frames[k][t] for t in tf.tolist()])}
        if states[k] is not None:
            ref.integrate(ev[used:][ev["t"][used:] <= t_end])
            got["S"], got["T"] = states[k]
            want = {"S": ref.S, "T": ref.T, "frames": ref_frames}
        else:
            # left: frames only (the state went with the stream)
            got["S"], got["T"] = np.zeros(1), np.zeros(1, dtype=np.int64)
            want = {"S": np.zeros(1), "T": np.zeros(1, dtype=np.int64), "frames": ref_frames}
        r = compare(got, want, p["C"], f"stream {k} {sp['W']}x{sp['H']}")
        worst["state_err"] = max(worst["state_err"], r["state_err"])
        worst["frame_max_lsb"] = max(worst["frame_max_lsb"], r["frame_max_lsb"])
        worst["frame_off_by_one"] += r["frame_off_by_one"]
        worst["frames"] += len(tf)
    return worst


def config3_specs(seconds=0.25):
    rates, streams = synth.serving_streams(64, seconds)
    specs = []
    for s in streams:
        specs.append(dict(W=s["W"], H=s["H"], events=synth.generate(s["scene"]),
                          arrivals=s["arrivals"], t_join_us=0, t_leave_us=None, tile_h=8))
    return specs


def test_64_stream_workload_matches_the_oracle_per_stream():
    t_end = 250_000
    specs = config3_specs(t_end / 1e6)
    assert sum(len(s["events"]) for s in specs) > 10_000_000
    frames, states, st = serve_schedule(specs, t_end)
    worst = check_against_oracle(specs, frames, states, t_end)
    assert worst["frames"] == 64 * 25
    assert st.streams_refused == 0
    print("64-stream workload:", worst)


def test_64_stream_workload_alone_equals_in_the_mix():
    t_end = 100_000
    specs = config3_specs(t_end / 1e6)
    mix_f, mix_s, _ = serve_schedule(specs, t_end)
    for k in (0, 17, 63):
        f, s, _ = serve_schedule([specs[k]], t_end)
        assert sorted(f[0]) == sorted(mix_f[k])
        for t in f[0]:
            assert np.array_equal(f[0][t], mix_f[k][t]), (k, t)
        assert np.array_equal(s[0][0], mix_s[k][0]) and np.array_equal(s[0][1], mix_s[k][1])


def test_mixed_resolution_workload_with_joins_and_leaves_matches_the_oracle():
    seconds = 0.25
    t_end = int(seconds * 1e6)
    ws = synth.mixed_serving(duration_s=seconds, counts=(4, 12, 32))
    arrs = synth.mixed_arrivals(ws, duration_s=seconds)
    tile_h = {2: 16, 1: 8, 0: 4}
    specs = [dict(W=w["W"], H=w["H"], events=synth.generate(w["scene"]), arrivals=a,
                  t_join_us=w["t_join_us"], t_leave_us=w["t_leave_us"], tile_h=tile_h[w["form"]])
             for w, a in zip(ws, arrs)]
    assert {s["W"] for s in specs} == {1280, 640, 346}
    assert any(s["t_join_us"] > 0 for s in specs) and any(s["t_leave_us"] for s in specs)
    frames, states, st = serve_schedule(specs, t_end)
    worst = check_against_oracle(specs, frames, states, t_end)
    assert st.streams_refused == 0
    print("mixed workload:", worst)
