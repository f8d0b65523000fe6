"""The tile kernel's segmented scan of clamped-affine event maps.

A pixel's events in one group of 32 due records can be composed instead of
applied one by one: every event is a monotone map S -> clamp(a S + b, lo, hi)
(Alg. 2 with the clamp of Eq. 13; Alg. 1 and Eq. 3 with exponential decay
without the clamp), and such maps compose associatively.  The scan runs for
groups in which one pixel holds at least `scan_chain` records (tuning; 33 is
off).  Its results must match the FP64 oracle within the parity tolerance
for every method, with the clamp binding or not, with ties in time, at every
threshold, and for per-event states; and it must run (results differ from
the event-by-event loop in the last bits where no clamp binds).
"""
import numpy as np
import pytest

import oracle
from esi_harness import (EXACT, GpuStream, compare, oracle_params, random_events, run_gpu,
                         run_oracle, state_error, STATE_TOL)

pytestmark = pytest.mark.gpu

BASE = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def hot_stream(seed, W, H, n, t1, hot_frac=0.5, n_hot=3):
    """Random events with n_hot very hot pixels in one tile row: groups of 32
    due records hold long same-pixel chains."""
    rng = np.random.default_rng(seed)
    ev = random_events(rng, W, H, n, 0, t1)
    sel = rng.random(n) < hot_frac
    k = rng.integers(0, n_hot, size=int(sel.sum()))
    ev["x"][sel] = (5 + 17 * k) % W
    ev["y"][sel] = 2 % H
    ev["p"][sel] = np.where(rng.random(int(sel.sum())) < 0.7, 1, -1)
    return ev


METHODS = [
    # (method, b, k, clamp, C): Alg. 2 with a binding clamp, Alg. 2 with
    # bounds that never bind, Alg. 1 (no clamp), Eq. 3 with exp decay, Eq. 2
    # (k = 0).  Eq. 2 takes a dyadic C: without decay a hot pixel's FP32 sum
    # of thousands of steps of 0.2 drifts from the FP64 sum (every addition
    # to a state near 800 rounds the same way), whichever order the sum takes;
    # with C = 0.25 every partial sum is exact, so the scan's regrouping must
    # give the oracle's value exactly
    (0, 2.0, 10.0, (-1.0, 1.0), 0.2),
    (0, 1.7, 50.0, (-40.0, 40.0), 0.2),
    (1, 2.0, 20.0, (-1.0, 1.0), 0.2),
    (2, 2.0, 30.0, (-1.0, 1.0), 0.2),
    (1, 2.0, 0.0, (-1.0, 1.0), 0.25),
    (0, 3.7, 1.0, (-0.5, 0.6), 0.2),
]


@pytest.mark.parametrize("method,b,k,clamp,C", METHODS)
@pytest.mark.parametrize("chain", [1, 2, 8, 32])
def test_scan_matches_the_oracle(method, b, k, clamp, C, chain):
    W, H = 150, 40
    ev = hot_stream(100 + method * 7 + chain, W, H, 60_000, 600_000)
    p = dict(BASE, C=C, method=method, b=b, k_per_s=k, s_min=clamp[0], s_max=clamp[1],
             render_decay=1)
    tf = np.arange(20_000, 600_001, 20_000)
    ref = run_oracle(ev, W, H, p, tf)
    got = run_gpu(ev, W, H, p, tf, tuning={"scan_chain": chain})
    compare(got, ref, p["C"], f"method {method} b={b} k={k} chain {chain}")
    if k == 0.0:
        assert np.array_equal(got["S"].astype(np.float64), ref["S"])


# Without a clamp an FP32 state that takes thousands of events between decays
# (k small, a pixel firing every few microseconds) drifts from the FP64 sum by
# more than 1e-5 whichever order it is summed in; the streams below keep the
# decay's memory to a few hundred events (k = 200 /s), where FP32 meets the
# bar and the scan's rounding can be compared with the loop's.
def test_scan_runs_and_rounds_like_the_loop():
    # no clamp and many events per pixel: the scan's products and sums round
    # in another order than the loop's, so some pixels differ in the last
    # bits, by no more than the loop's own distance from the oracle
    W, H = 150, 40
    ev = hot_stream(7, W, H, 80_000, 400_000, hot_frac=0.8)
    p = dict(BASE, method=1, k_per_s=200.0, render_decay=1)
    tf = np.arange(50_000, 400_001, 50_000)
    loop = run_gpu(ev, W, H, p, tf, tuning=EXACT)
    scan = run_gpu(ev, W, H, p, tf, tuning={"scan_chain": 2})
    ref = run_oracle(ev, W, H, p, tf)
    e_loop = compare(loop, ref, p["C"], "loop")["state_err"]
    e_scan = compare(scan, ref, p["C"], "scan")["state_err"]
    assert not np.array_equal(loop["S"], scan["S"])
    assert np.array_equal(loop["T"], scan["T"])
    assert e_scan <= 4 * e_loop + 1e-7, (e_scan, e_loop)


def test_scan_with_ties_and_a_binding_clamp_keeps_arrival_order():
    # equal times at one pixel (d = 1): only the clamp makes the order matter;
    # the scan composes in arrival order
    from synth import EVENT_DTYPE
    W, H = 64, 8
    rows = []
    t = 1000
    for g in range(200):
        t += 137
        for j in range(30):
            rows.append((t, 3, 1, 1 if (j + g) % 5 else -1))
        rows.append((t, 9, 2, 1))
    ev = np.zeros(len(rows), dtype=EVENT_DTYPE)
    for i, (tt, x, y, pol) in enumerate(rows):
        ev[i]["t"], ev[i]["x"], ev[i]["y"], ev[i]["p"] = tt, x, y, pol
    for clamp in ((-0.3, 0.5), (-1.0, 1.0)):
        p = dict(BASE, C=0.15, k_per_s=100.0, s_min=clamp[0], s_max=clamp[1], render_decay=1)
        tf = np.array([int(ev["t"][-1])], dtype=np.int64)
        ref = run_oracle(ev, W, H, p, tf)
        compare(run_gpu(ev, W, H, p, tf, tuning={"scan_chain": 1}), ref, p["C"], str(clamp))


@pytest.mark.parametrize("method", [0, 1, 2])
def test_scan_per_event_states(method):
    W, H = 130, 30
    ev = hot_stream(55 + method, W, H, 40_000, 300_000)
    p = dict(BASE, method=method, k_per_s=200.0)
    st = oracle.OracleState(W, H, oracle_params(p))
    ref = st.event_states(ev)
    with GpuStream(W, H, p, {"scan_chain": 2}) as g:
        g.esi.check(g.push(ev), "push")
        import torch
        out = torch.empty(len(ev), dtype=torch.float32, device="cuda")
        rc, m = g.esi.esi_event_states(g.h, out, len(ev), 1)
        g.esi.check(rc, "event_states")
        got = out.cpu().numpy().astype(np.float64)
        assert m == len(ev)
        den = np.maximum(np.abs(ref), p["C"])
        assert np.max(np.abs(got - ref) / den) <= STATE_TOL
        S, T = g.state()
        assert np.array_equal(T, st.T)
        assert state_error(S, st.S, p["C"]) <= STATE_TOL


def test_scan_chain_knob_validation():
    from paper_2508_02238_gb300 import esi
    with GpuStream(64, 32, dict(BASE)) as g:
        t = esi.esi_tuning()
        for bad in (-1, 34, 1000):
            t.scan_chain = bad
            assert esi.esi_set_tuning(g.h, t) == esi.ESI_EINVAL
        t.scan_chain = 0
        assert esi.esi_set_tuning(g.h, t) == 0
        rc, got = esi.esi_get_tuning(g.h)
        assert rc == 0 and got.scan_chain == 8
    opts = esi.esi_server_opts()
    opts.scan_chain = 34
    rc, srv = esi.esi_server_create(1 << 20, opts, 0)
    assert rc == esi.ESI_EINVAL
