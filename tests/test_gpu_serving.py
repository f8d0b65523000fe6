"""Batched serving (esi_server_*) against the oracle and the single-sensor path.

Each stream of a server must give, frame for frame, what the oracle gives
for that stream alone (parity tolerance of esi_harness), and exactly what it
gives when served alone: streams never interact.
"""
import numpy as np
import pytest

import oracle
import synth
from esi_harness import GpuStream, compare, oracle_params, random_events, run_oracle

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
]


def make_stream_events(i, W, H, p, kind, t_end):
    t0 = p.get("t_origin_us", 0)
    if kind == "sinusoid":
        sc = synth.serving_stream(i, 2.0e6, (t_end - t0) / 1e6, W=W, H=H, t0_us=t0)
        return synth.generate(sc)
    rng = np.random.default_rng(100 + i)
    return random_events(rng, W, H, int(0.5 * W * H * (t_end - t0) / 1e5), t0, t_end,
                         hot=(W // 3, H // 2, 0.02))


def drive(esi, srv, ids, events, dims, t_end, tick_us=1000, start=0):
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
        assert esi.esi_server_tick(srv, now) == 0
        assert esi.esi_server_sync(srv) == 0
        for sid in ids:
            W, H = dims[sid]
            out = outs.setdefault(sid, np.empty((H, W), dtype=np.uint8))
            rc, tf, lat = esi.esi_stream_frame(srv, sid, out)
            if rc == 0:
                frames[sid][tf] = out.copy()
    return frames


def serve(stream_specs, t_end, use_graph=1, budget=256 << 20):
    esi = _esi()
    opts = esi.esi_server_opts()
    opts.use_graph = use_graph
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
        frames = drive(esi, srv, ids, events, dims, t_end)
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
    W, H, p, kind = STREAMS[1]
    t_end = 100_000
    res, _ = serve([(1, STREAMS[1])], t_end)
    frames, (S, T), ev = res[1]
    tf = sorted(frames)
    used = ev[ev["t"] <= t_end]
    with GpuStream(W, H, {**dict(t_origin_us=0), **p}) as g:
        assert g.push(used) == 0
        rc, fr = g.render_frames(tf)
        assert rc == 0
        rc, _ = g.render_frame(t_end)   # the server has applied everything up to t_end
        assert rc == 0
        Sh, Th = g.state()
    assert np.array_equal(np.stack([frames[t] for t in tf]), fr)
    assert np.array_equal(S, Sh) and np.array_equal(T, Th)


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
