"""Continuous-time output (esi_event_states) against the oracle.

Each value is a state, so the state tolerance of esi_harness applies to it
(1e-5 relative, floor C); NaN marks the same events (outside the sensor) on
both sides.  The state left behind is bit-identical to a render's.
"""
import numpy as np
import pytest

import oracle
from esi_harness import EXACT, GpuStream, STATE_TOL, oracle_params, random_events, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def P(**kw):
    d = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-0.8, s_max=1.2)
    d.update(kw)
    return d


def check_values(got, ref, C, label=""):
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan), label
    den = np.maximum(np.abs(ref[~nan]), C)
    err = np.max(np.abs(got[~nan].astype(np.float64) - ref[~nan]) / den) if (~nan).any() else 0.0
    assert err <= STATE_TOL, f"{label}: per-event err {err:.3e}"


def gpu_event_states(g, n, on_device=False):
    import torch
    if on_device:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        rc, m = g.esi.esi_event_states(g.h, out, n, 1)
        g.esi.check(rc, "event_states")
        return out.cpu().numpy(), m
    out = np.empty(n, dtype=np.float32)
    rc, m = g.esi.esi_event_states(g.h, out, n, 0)
    g.esi.check(rc, "event_states")
    return out, m


TUNINGS = [None, dict(tile_w=32, tile_h=16), dict(tile_w=64, tile_h=8),
           dict(tile_h=4, chunk_events=512, batch_records=1024, max_batch_events=4096)]


@pytest.mark.parametrize("W,H", [(100, 70), (346, 260), (37, 19)])
@pytest.mark.parametrize("method,b,k", [(0, 2.0, 10.0), (0, 1.7, 30.0), (1, 2.0, 10.0),
                                         (1, 2.0, 0.0), (2, 2.0, 50.0)])
@pytest.mark.parametrize("ti", range(len(TUNINGS)))
def test_event_states_match_the_oracle(W, H, method, b, k, ti):
    rng = np.random.default_rng(W * 7 + H + int(k) + 11 * method + ti)
    ev = random_events(rng, W + 1, H, 20_000, 0, 400_000, hot=(W // 2, H // 3, 0.05))
    p = P(method=method, b=b, k_per_s=k)
    st = oracle.OracleState(W, H, oracle_params(p))
    ref = st.event_states(ev)
    with GpuStream(W, H, p, TUNINGS[ti]) as g:
        g.esi.check(g.push(ev), "push")
        got, m = gpu_event_states(g, len(ev), on_device=bool(ti % 2))
        assert m == len(ev)
        check_values(got, ref, p["C"], f"{W}x{H} m={method} t={ti}")
        S, T = g.state()
        assert np.array_equal(T, st.T)
        den = np.maximum(np.abs(st.S), p["C"])
        assert np.max(np.abs(S - st.S) / den) <= STATE_TOL
        assert g.stats().events_pending == 0


@pytest.mark.parametrize("method", [0, 2])
def test_state_after_event_states_equals_a_render(method):
    rng = np.random.default_rng(90 + method)
    W, H = 200, 150
    ev = random_events(rng, W, H, 80_000, 0, 800_000, hot=(33, 40, 0.1))
    p = P(method=method, render_decay=1)
    # with the scan off (it composes each group in its own rounding, and the
    # per-event walk groups records without frame boundaries)
    for tun in (EXACT, dict(tile_h=16, chunk_events=1024, max_batch_events=10_000, **EXACT)):
        r = run_gpu(ev, W, H, p, [int(ev["t"][-1])], tuning=tun)
        with GpuStream(W, H, p, tun) as g:
            g.esi.check(g.push(ev), "push")
            gpu_event_states(g, len(ev))
            S, T = g.state()
        assert np.array_equal(S, r["S"]) and np.array_equal(T, r["T"])


def test_event_states_then_frames_and_more_events():
    # events A -> per-event states; events B -> frames: the same as the
    # oracle applying A then B
    rng = np.random.default_rng(95)
    W, H = 130, 90
    A = random_events(rng, W, H, 30_000, 0, 300_000, hot=(5, 7, 0.05))
    B = random_events(rng, W, H, 30_000, 300_000, 600_000, hot=(5, 7, 0.05))
    p = P(render_decay=1)
    st = oracle.OracleState(W, H, oracle_params(p))
    ref_vals = st.event_states(A)
    tf = np.arange(350_000, 600_001, 50_000)
    ref_frames, _ = st.replay(B, tf)
    with GpuStream(W, H, p) as g:
        g.esi.check(g.push(A), "push A")
        vals, _ = gpu_event_states(g, len(A))
        check_values(vals, ref_vals, p["C"])
        # a frame before the last applied event is refused
        rc, _ = g.render_frame(int(A["t"][-1]) - 1)
        assert rc == g.esi.ESI_ETIMEORDER
        g.esi.check(g.push(B), "push B")
        rc, frames = g.render_frames(tf)
        g.esi.check(rc, "render")
        d = np.abs(frames.astype(np.int16) - ref_frames.astype(np.int16))
        assert d.max() <= 1
        S, T = g.state()
        assert np.array_equal(T, st.T)


def test_event_states_edge_cases():
    W, H = 16, 8
    p = P()
    with GpuStream(W, H, p) as g:
        out = np.full(4, 7.0, dtype=np.float32)
        rc, m = g.esi.esi_event_states(g.h, out, 4, 0)
        assert rc == 0 and m == 0 and np.all(out == 7.0)
        ev = random_events(np.random.default_rng(1), W, H, 10, 0, 1000)
        g.esi.check(g.push(ev), "push")
        rc, m = g.esi.esi_event_states(g.h, out, 4, 0)
        assert rc == g.esi.ESI_ERANGE and m == 10
        assert g.stats().events_pending == 10
    # a time span beyond 32 bits splits into sub-batches
    rng = np.random.default_rng(2)
    ev = random_events(rng, W, H, 5000, 0, 3 * 2**32)
    p = P(k_per_s=1e-4, b=1.5)
    st = oracle.OracleState(W, H, oracle_params(p))
    ref = st.event_states(ev)
    with GpuStream(W, H, p) as g:
        g.esi.check(g.push(ev), "push")
        got, _ = gpu_event_states(g, len(ev), on_device=True)
    check_values(got, ref, p["C"], "span > 2^32 us")
