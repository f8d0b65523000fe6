"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

None of these re-types the oracle's loop: each compares it with a different
formulation (Eq. 2, the corrected Eq. 5 product form, the Eq. 6 inequality,
hand-worked numbers, symmetry and independence properties, or a fold of the
clamped-affine maps in every bracketing).  A dropped term, a wrong sign, a
transposed operand or a misplaced clamp fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import OracleParams, OracleState
from synth import EVENT_DTYPE


def make_events(rows):
    """rows: iterable of (t, x, y, p)."""
    rows = list(rows)
    ev = np.zeros(len(rows), dtype=EVENT_DTYPE)
    for i, (t, x, y, p) in enumerate(rows):
        ev[i]["t"], ev[i]["x"], ev[i]["y"], ev[i]["p"] = t, x, y, p
    return ev


def random_stream(rng, W, H, n, t_max, pol_bias=0.5):
    t = np.sort(rng.integers(0, t_max, size=n))
    ev = np.zeros(n, dtype=EVENT_DTYPE)
    ev["t"] = t
    ev["x"] = rng.integers(0, W, size=n)
    ev["y"] = rng.integers(0, H, size=n)
    ev["p"] = np.where(rng.random(n) < pol_bias, 1, -1)
    return ev


BIG = 1e30  # clamp bounds that never bind: Alg. 1 (no clamp) behaviour


def d_np(dt_us, k_per_s, b):
    """Eq. 4 written independently with numpy (reading max(1 - k t, 0)^b)."""
    u = 1.0 - (k_per_s * 1e-6) * np.asarray(dt_us, dtype=np.float64)
    return np.where(u > 0.0, np.maximum(u, 0.0) ** b, 0.0)


# ----------------------------------------------------------------- Eq. 4 / Eq. 6
@pytest.mark.parametrize("k", [0.5, 10.0, 100.0, 1e4])
@pytest.mark.parametrize("b", [0.5, 1.0, 2.0, 3.7])
def test_decay_endpoints_monotone(k, b):
    assert oracle.decay(0, k, b) == 1.0                      # d(0) = 1
    cutoff = 1.0 / (k * 1e-6)
    assert oracle.decay(int(np.ceil(cutoff)) + 1, k, b) == 0.0  # k t >= 1 -> 0
    assert oracle.decay(int(10 * cutoff), k, b) == 0.0
    assert oracle.decay(max(int(cutoff) - 1, 1), k, b) > 0.0
    ts = np.unique(np.linspace(0, 1.2 * cutoff, 400).astype(np.int64))
    vals = np.array([oracle.decay(int(t), k, b) for t in ts])
    assert np.all(np.diff(vals) <= 0.0)                     # non-increasing
    assert np.all((vals >= 0.0) & (vals <= 1.0))


def test_decay_k_zero_is_one():
    # k = 0 turns Eq. 3/Alg. 2 into the plain integration of Eq. 2
    for dt in (0, 1, 10**6, 10**12):
        assert oracle.decay(dt, 0.0, 2.0) == 1.0


@pytest.mark.parametrize("k", [10.0, 1000.0])
@pytest.mark.parametrize("b", [0.5, 1.0, 2.0, 3.7])
@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_decay_eq6_inequality(k, b, n):
    # Eq. 6: d(t)^n > d(n t) for 0 < t < 1/(n k), n >= 2 (proved by Eq. 7-12)
    lim = 1.0 / (n * k * 1e-6)
    for t in np.unique(np.linspace(1, lim - 1, 60).astype(np.int64)):
        if t <= 0 or t >= lim:
            continue
        assert oracle.decay(int(t), k, b) ** n > oracle.decay(int(n * t), k, b)


# ------------------------------------------------------- hand-worked examples
# k = 1e5 /s means k = 0.1 per microsecond, so d(dt) = max(1 - dt/10, 0)^b.
HAND = dict(k_per_s=1e5)


def test_hand_single_event():
    # one +1 event at t = 5 us: S = C d(5) = 0.5 * 0.5^2 = 0.125 (b = 2)
    p = OracleParams(C=0.5, b=2.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(3, 2, p)
    st.integrate(make_events([(5, 1, 1, 1)]))
    S = st.S.reshape(2, 3)
    assert S[1, 1] == pytest.approx(0.125, rel=1e-15)
    assert np.count_nonzero(st.S) == 1
    assert st.T.reshape(2, 3)[1, 1] == 5 and np.count_nonzero(st.T) == 1


def test_hand_single_event_after_cutoff_contributes_nothing():
    # an event after >= 1/k of silence is multiplied by d = 0 (add-then-decay order)
    p = OracleParams(C=0.5, b=2.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(2, 2, p)
    # (gaps of 11 and 26 us exceed 1/k = 10 us; exactly 10 us leaves u ~ 1e-16
    # because k * 1e-6 is not exact in binary)
    st.integrate(make_events([(11, 0, 0, 1), (26, 1, 0, -1)]))
    assert st.S[0] == 0.0 and st.S[1] == 0.0
    assert st.T[0] == 11 and st.T[1] == 26


def test_hand_two_events_same_pixel():
    # b = 1: events (+, t=2), (-, t=7) at one pixel, origin 0, clamp [-1, 1]
    #   S1 = (0 + 0.5)(1 - 0.2) = 0.4
    #   S2 = (0.4 - 0.5)(1 - 0.5) = -0.05
    p = OracleParams(C=0.5, b=1.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(1, 1, p)
    st.integrate(make_events([(2, 0, 0, 1), (7, 0, 0, -1)]))
    assert st.S[0] == pytest.approx(-0.05, rel=1e-14)
    # tight clamp [-0.02, 0.3]: S1 = min(0.4, 0.3) = 0.3; S2 = (0.3 - 0.5)*0.5 = -0.1 -> -0.02
    p2 = OracleParams(C=0.5, b=1.0, s_min=-0.02, s_max=0.3, **HAND)
    st2 = OracleState(1, 1, p2)
    st2.integrate(make_events([(2, 0, 0, 1)]))
    assert st2.S[0] == pytest.approx(0.3, rel=1e-15)
    st2.integrate(make_events([(7, 0, 0, -1)]))
    assert st2.S[0] == pytest.approx(-0.02, rel=1e-15)


def test_hand_ties_same_time():
    # two +1 events at t = 5 at one pixel: the second sees dt = 0, d = 1
    #   C = 0.6, b = 1: S1 = 0.6 * 0.5 = 0.3, S2 = 0.3 + 0.6 = 0.9
    p = OracleParams(C=0.6, b=1.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(1, 1, p)
    st.integrate(make_events([(5, 0, 0, 1), (5, 0, 0, 1)]))
    assert st.S[0] == pytest.approx(0.9, rel=1e-14)
    #   C = 0.8: S1 = 0.4, S2 = 1.2 -> clamped to 1.0 (Eq. 13)
    p = OracleParams(C=0.8, b=1.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(1, 1, p)
    st.integrate(make_events([(5, 0, 0, 1), (5, 0, 0, 1)]))
    assert st.S[0] == 1.0


def test_polarity_reading():
    # p > 0 -> +1, otherwise -1 (accepts DAVIS 0/1 polarity as well as +-1)
    p = OracleParams(C=0.5, b=1.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(3, 1, p)
    st.integrate(make_events([(5, 0, 0, 1), (5, 1, 0, 0), (5, 2, 0, -1)]))
    assert st.S[0] == pytest.approx(0.25, rel=1e-15)
    assert st.S[1] == pytest.approx(-0.25, rel=1e-15)
    assert st.S[2] == pytest.approx(-0.25, rel=1e-15)


# -------------------------------------------------------------------- Eq. 14
def test_render_hand_values():
    p = OracleParams(C=0.5, b=2.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(4, 1, p)
    st.S[:] = [-1.0, 1.0, 0.0, 0.25]
    st.T[:] = 0
    B = st.render(0, render_decay=0).ravel()
    # 255*(S+1)/2: 0, 255, 127.5 -> 128 (half to even), 159.375 -> 159
    assert list(B) == [0, 255, 128, 159]
    # decay view at t = 5: d = 0.5^2 = 0.25; S=1 -> 0.25 -> 159
    st.S[:] = 1.0
    B = st.render(5, render_decay=1).ravel()
    assert list(B) == [159, 159, 159, 159]
    # the view is not written back
    assert np.all(st.S == 1.0)
    # after the cutoff the view is 0 -> 128
    assert list(st.render(10, render_decay=1).ravel()) == [128] * 4


def test_zero_events_frame():
    # no events: S = 0, T = t_origin everywhere; B = rint(255 (0 - Smin)/(Smax - Smin))
    p = OracleParams(C=0.2, k_per_s=10.0, b=2.0, s_min=-0.5, s_max=1.5,
                     t_origin_us=123)
    st = OracleState(7, 5, p)
    assert np.all(st.S == 0.0) and np.all(st.T == 123)
    for rd in (0, 1):
        B = st.render(10_000, render_decay=rd)
        assert np.all(B == 64)  # 255 * 0.5 / 2 = 63.75 -> 64


# -------------------------------------------------------------------- Eq. 2
def test_eq2_plain_integration_when_k_is_zero():
    # k = 0: d = 1 and with non-binding bounds S = C (n_plus - n_minus) exactly
    rng = np.random.default_rng(1)
    W, H = 9, 7
    ev = random_stream(rng, W, H, 4000, 10**6)
    p = OracleParams(C=0.25, k_per_s=0.0, b=2.0, s_min=-BIG, s_max=BIG)
    st = OracleState(W, H, p)
    st.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    sgn = np.where(ev["p"] > 0, 1, -1)
    net = np.bincount(pix, weights=sgn, minlength=W * H)
    assert np.array_equal(st.S, 0.25 * net)
    last = np.zeros(W * H, dtype=np.int64)
    last[pix] = ev["t"]          # later assignment wins: last event per pixel
    assert np.array_equal(st.T, last)


# ------------------------------------------------------ corrected Eq. 5 form
@pytest.mark.parametrize("b", [0.5, 1.0, 2.0, 3.7])
@pytest.mark.parametrize("k", [1.0, 10.0, 100.0])
def test_eq5_closed_form_clamp_free(b, k):
    # S_n = C sum_i s_i prod_{j=i..n} d(t_j - t_{j-1}), t_0 = T_init (no clamp)
    rng = np.random.default_rng(int(b * 10 + k))
    W, H = 8, 6
    t_origin = 1000
    ev = random_stream(rng, W, H, 3000, 400_000)
    ev["t"] += t_origin
    p = OracleParams(C=0.3, k_per_s=k, b=b, s_min=-BIG, s_max=BIG,
                     t_origin_us=t_origin)
    st = OracleState(W, H, p)
    st.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for q in range(W * H):
        sel = ev[pix == q]
        if len(sel) == 0:
            assert st.S[q] == 0.0 and st.T[q] == t_origin
            continue
        t = np.concatenate([[t_origin], sel["t"]])
        a = d_np(np.diff(t), k, b)                  # a_j = d(t_j - t_{j-1})
        suffix = np.cumprod(a[::-1])[::-1]          # prod_{j=i..n} a_j
        s = np.where(sel["p"] > 0, 1.0, -1.0)
        expect = 0.3 * np.sum(s * suffix)
        assert st.S[q] == pytest.approx(expect, rel=1e-11, abs=1e-15)
        assert st.T[q] == sel["t"][-1]


# ---------------------------------------------------------------- symmetries
def test_superposition_clamp_free():
    rng = np.random.default_rng(5)
    W, H = 6, 5
    ev = random_stream(rng, W, H, 3000, 300_000)
    base = OracleParams(C=0.2, k_per_s=20.0, b=1.7, s_min=-BIG, s_max=BIG)
    ref = OracleState(W, H, base)
    ref.integrate(ev)
    # negating every polarity negates S (the update is linear in p_i C)
    neg = ev.copy()
    neg["p"] = -neg["p"]
    st = OracleState(W, H, base)
    st.integrate(neg)
    assert np.array_equal(st.S, -ref.S)
    # scaling C by 2 scales S by 2 exactly; by 3 up to rounding
    for lam, tol in ((2.0, 0.0), (3.0, 1e-13)):
        p2 = OracleParams(C=0.2 * lam, k_per_s=20.0, b=1.7, s_min=-BIG, s_max=BIG)
        st = OracleState(W, H, p2)
        st.integrate(ev)
        if tol == 0.0:
            assert np.array_equal(st.S, lam * ref.S)
        else:
            assert np.allclose(st.S, lam * ref.S, rtol=tol, atol=1e-15)
    assert np.array_equal(st.T, ref.T)


def test_pixel_independence_under_reordering():
    # the result depends only on each pixel's own time-ordered events
    rng = np.random.default_rng(7)
    W, H = 10, 4
    ev = random_stream(rng, W, H, 5000, 200_000)
    p = OracleParams(C=0.35, k_per_s=15.0, b=2.5, s_min=-0.7, s_max=0.9)
    a = OracleState(W, H, p)
    a.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for order in (np.argsort(pix, kind="stable"),
                  np.argsort(-pix, kind="stable"),
                  np.argsort(pix % 3, kind="stable")):
        b = OracleState(W, H, p)
        b.integrate(ev[order])
        assert np.array_equal(a.S, b.S) and np.array_equal(a.T, b.T)


def test_frames_do_not_change_state():
    # rendering (with or without the decay view) never writes S or T back,
    # so any split into windows ends in the same state
    rng = np.random.default_rng(9)
    W, H = 12, 9
    ev = random_stream(rng, W, H, 6000, 500_000)
    for rd in (0, 1):
        p = OracleParams(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0,
                         render_decay=rd)
        one = OracleState(W, H, p)
        one.integrate(ev)
        many = OracleState(W, H, p)
        frames, used = many.replay(ev, np.arange(10_000, 500_001, 10_000))
        assert used == len(ev)
        assert np.array_equal(one.S, many.S) and np.array_equal(one.T, many.T)
        # frame w equals a render after integrating exactly the events t <= t_w
        tw = 250_000
        pre = OracleState(W, H, p)
        pre.integrate(ev[ev["t"] <= tw])
        assert np.array_equal(frames[24], pre.render(tw))


def test_clamp_bounds_hold():
    rng = np.random.default_rng(11)
    W, H = 5, 5
    ev = random_stream(rng, W, H, 20000, 100_000, pol_bias=0.8)
    p = OracleParams(C=0.3, k_per_s=5.0, b=2.0, s_min=-0.4, s_max=0.6)
    st = OracleState(W, H, p)
    st.integrate(ev)
    assert np.all(st.S >= -0.4) and np.all(st.S <= 0.6)
    assert np.any(st.S == 0.6)  # hot positive pixels saturate (Eq. 13)


def test_out_of_range_events_dropped():
    p = OracleParams(C=0.5, b=1.0, s_min=-1.0, s_max=1.0, **HAND)
    st = OracleState(3, 2, p)
    used = st.integrate(make_events([(1, 3, 0, 1), (2, 0, 2, 1), (3, 2, 1, 1)]))
    assert used == 1 and st.dropped[0] == 2
    assert np.count_nonzero(st.S) == 1 and st.T.reshape(2, 3)[1, 2] == 3


# ----------------------------------------- brute force: clamped-affine folds
def compose(g, f):
    """g after f for maps x -> clamp(a x + beta, L, H) with a >= 0."""
    a1, b1, L1, H1 = f
    a2, b2, L2, H2 = g
    return (a2 * a1, a2 * b1 + b2,
            np.clip(a2 * L1 + b2, L2, H2), np.clip(a2 * H1 + b2, L2, H2))


def bracketings(elems):
    """Every binary bracketing of the ordered list of maps, composed."""
    if len(elems) == 1:
        return [elems[0]]
    out = []
    for split in range(1, len(elems)):
        for left in bracketings(elems[:split]):
            for right in bracketings(elems[split:]):
                out.append(compose(right, left))
    return out


@pytest.mark.parametrize("b", [1.0, 2.5])
@pytest.mark.parametrize("bounds", [(-0.3, 0.5), (-BIG, BIG), (0.1, 0.2)])
def test_bruteforce_clamped_affine_fold(b, bounds):
    # all sequences of <= 4 events over {2 pixels x 2 polarities x 3 gaps}
    # (gaps 0, 40 us and 150 us >= 1/k with k = 1e4 /s); every sequence sits on
    # its own 2 pixels of a 2-wide sensor, then all are merged in time order.
    k = 1e4
    C = 0.35
    L, Hb = bounds
    gaps = (0, 40, 150)
    alphabet = list(itertools.product((0, 1), (1, -1), gaps))
    seqs = [s for n in range(1, 5) for s in itertools.product(alphabet, repeat=n)]
    rows = []
    for r, seq in enumerate(seqs):
        t = 0
        for (px, pol, gap) in seq:
            t += gap
            rows.append((t, px, r, pol))
    rows.sort(key=lambda e: e[0])       # stable: keeps each sequence's order
    ev = make_events(rows)
    p = OracleParams(C=C, k_per_s=k, b=b, s_min=L, s_max=Hb)
    st = OracleState(2, len(seqs), p)
    st.integrate(ev)
    S = st.S.reshape(len(seqs), 2)
    # group pixels by their event count and fold vectorised over sequences
    per_pixel = {}
    for r, seq in enumerate(seqs):
        t = 0
        lists = ([], [])
        for (px, pol, gap) in seq:
            t += gap
            lists[px].append((t, pol))
        for px in (0, 1):
            per_pixel.setdefault(len(lists[px]), []).append((r, px, lists[px]))
    checked = 0
    for m, items in per_pixel.items():
        if m == 0:
            for r, px, _ in items:
                assert S[r, px] == 0.0
            continue
        ts = np.array([[0] + [e[0] for e in lst] for _, _, lst in items], dtype=np.int64)
        pols = np.array([[e[1] for e in lst] for _, _, lst in items], dtype=np.float64)
        a = d_np(np.diff(ts, axis=1), k, b)              # (N, m)
        elems = [(a[:, i], a[:, i] * pols[:, i] * C,
                  np.full(len(items), L), np.full(len(items), Hb)) for i in range(m)]
        got = np.array([S[r, px] for r, px, _ in items])
        for comp in bracketings(elems):
            aa, bb, LL, HH = comp
            val = np.clip(aa * 0.0 + bb, LL, HH)       # applied to S = 0
            assert np.allclose(val, got, rtol=1e-12, atol=1e-12)
            checked += 1
    assert checked == 9  # 1 + 1 + 2 + 5 bracketings for pixel sequences of 1..4 events


# --------------------------------------------- brute force on a 4x4 sensor
@pytest.mark.parametrize("bounds", [(-BIG, BIG), (-0.3, 0.45)])
def test_bruteforce_every_event_pair_on_a_4x4_sensor(bounds):
    # every ordered pair of events on its own 4x4 sensor: first event at any
    # pixel, either polarity, at t = 0 or 30 us; second at any pixel, either
    # polarity, 0, 40 or 600 us later (k = 2e3 /s: 600 us is past the decay's
    # cutoff of 500 us).  Each pixel's S and T against its own events composed
    # as clamped-affine maps, and the decay-view frame at the last event's
    # time against Eq. 14 applied to that, for every one of the 16 positions
    # (x, y swapped or an index off by one fails here).
    k, b, C = 2e3, 2.0, 0.35
    L, Hb = bounds
    p = OracleParams(C=C, k_per_s=k, b=b, s_min=L, s_max=Hb)
    firsts = list(itertools.product(range(16), (1, -1), (0, 30)))
    seconds = list(itertools.product(range(16), (1, -1), (0, 40, 600)))
    cases = [(f,) for f in firsts] + [(f, s) for f in firsts for s in seconds]
    for case in cases:
        rows, t = [], 0
        for j, ev in enumerate(case):
            q, pol, dt = ev
            t = dt if j == 0 else t + dt
            rows.append((t, q % 4, q // 4, pol))
        st = OracleState(4, 4, p)
        st.integrate(make_events(rows))
        t_f = rows[-1][0]
        frame = st.render(t_f, render_decay=1).ravel()
        for q in range(16):
            mine = [(t, pol) for (t, x, y, pol) in rows if y * 4 + x == q]
            if not mine:
                assert st.S[q] == 0.0 and st.T[q] == 0
                expect_s, expect_t = 0.0, 0
            else:
                ts = np.array([0] + [e[0] for e in mine], dtype=np.int64)
                a = d_np(np.diff(ts), k, b)
                maps = [(a[i], a[i] * mine[i][1] * C, L, Hb) for i in range(len(mine))]
                m = maps[0]
                for g in maps[1:]:
                    m = compose(g, m)
                expect_s = float(np.clip(m[0] * 0.0 + m[1], m[2], m[3]))
                expect_t = mine[-1][0]
                assert st.S[q] == pytest.approx(expect_s, rel=1e-12, abs=1e-15), (case, q)
                assert st.T[q] == expect_t, (case, q)
            if Hb < BIG:
                view = expect_s * float(d_np(t_f - expect_t, k, b))
                u = 255.0 * (view - L) / (Hb - L)
                if abs(u - np.floor(u) - 0.5) > 1e-9:     # away from a rounding tie
                    assert frame[q] == np.clip(np.rint(u), 0, 255), (case, q)
                else:
                    assert abs(int(frame[q]) - float(u)) <= 0.5 + 1e-9, (case, q)
    assert len(cases) == 64 + 64 * 96


# ------------------------------------------- Alg. 1 and Eq. 3 as methods
def eq3_direct(ev_pix, t, k, C):
    """Eq. 3 with d(t) = exp(-k t), summed term by term at time t (events t_i <= t)."""
    sel = ev_pix[ev_pix["t"] <= t]
    s = np.where(sel["p"] > 0, 1.0, -1.0)
    return C * float(np.sum(s * np.exp(-(k * 1e-6) * (t - sel["t"]).astype(np.float64))))


@pytest.mark.parametrize("b", [0.5, 2.0])
def test_alg1_is_the_clamp_free_loop(b):
    # Alg. 1 has no clamp: with bounds that bind for Alg. 2 the Alg. 1 state
    # still follows the corrected Eq. 5 product form, and Alg. 2 differs
    rng = np.random.default_rng(31)
    W, H, k, C = 5, 4, 5.0, 0.3
    ev = random_stream(rng, W, H, 4000, 300_000, pol_bias=0.8)
    p1 = OracleParams(C=C, k_per_s=k, b=b, s_min=-0.3, s_max=0.3, method=1)
    p2 = OracleParams(C=C, k_per_s=k, b=b, s_min=-0.3, s_max=0.3, method=0)
    a1, a2 = OracleState(W, H, p1), OracleState(W, H, p2)
    a1.integrate(ev)
    a2.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for q in range(W * H):
        sel = ev[pix == q]
        t = np.concatenate([[0], sel["t"]])
        suffix = np.cumprod(d_np(np.diff(t), k, b)[::-1])[::-1]
        expect = C * np.sum(np.where(sel["p"] > 0, 1.0, -1.0) * suffix)
        assert a1.S[q] == pytest.approx(expect, rel=1e-11, abs=1e-15)
    assert np.max(np.abs(a1.S)) > 0.6          # the bounds would have bound
    assert np.all((a2.S >= -0.3) & (a2.S <= 0.3))
    assert np.array_equal(a1.T, a2.T)


@pytest.mark.parametrize("method", [1, 2])
def test_k_zero_is_eq2_for_unclamped_methods(method):
    # Alg. 1 and Eq. 3 with k = 0 are Eq. 2: S = C (n_plus - n_minus), even
    # with narrow bounds (neither method clamps)
    rng = np.random.default_rng(32 + method)
    W, H = 7, 6
    ev = random_stream(rng, W, H, 5000, 10**6, pol_bias=0.7)
    p = OracleParams(C=0.25, k_per_s=0.0, b=2.0, s_min=-0.5, s_max=0.5, method=method)
    st = OracleState(W, H, p)
    st.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    net = np.bincount(pix, weights=np.where(ev["p"] > 0, 1, -1), minlength=W * H)
    assert np.array_equal(st.S, 0.25 * net)
    assert np.max(np.abs(st.S)) > 0.5


@pytest.mark.parametrize("k", [1.0, 10.0, 300.0])
def test_eq3_exp_matches_the_direct_sum(k):
    # the regrouped recurrence equals Eq. 3's sum over every past event, at
    # the last event (the state) and at each frame time (the decay view)
    rng = np.random.default_rng(int(k) + 40)
    W, H, C = 6, 5, 0.2
    ev = random_stream(rng, W, H, 3000, 500_000)
    tf = np.array([120_000, 250_001, 400_000, 500_000], dtype=np.int64)
    lo, hi = -1.5, 2.0
    p = OracleParams(C=C, k_per_s=k, b=7.0, s_min=lo, s_max=hi, render_decay=1, method=2)
    st = OracleState(W, H, p)
    frames, used = st.replay(ev, tf)
    assert used == len(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for q in range(W * H):
        ev_q = ev[pix == q]
        if len(ev_q):
            assert st.S[q] == pytest.approx(eq3_direct(ev_q, ev_q["t"][-1], k, C),
                                             rel=1e-11, abs=1e-15)
        for w, t in enumerate(tf):
            x = 255.0 * (eq3_direct(ev_q, t, k, C) - lo) / (hi - lo)
            if abs(x - np.floor(x) - 0.5) > 1e-6:     # away from a rounding tie
                assert frames[w].ravel()[q] == int(np.clip(np.rint(x), 0, 255))


def test_eq3_exp_decay_is_exp():
    for dt, k in ((0, 10.0), (1, 10.0), (100_000, 10.0), (7, 1e4), (10**9, 1e-3)):
        assert oracle.decay_exp(dt, k) == pytest.approx(np.exp(-k * 1e-6 * dt), rel=1e-15)
    assert oracle.decay_exp(0, 123.0) == 1.0


def first_event_residual(method, gaps_us, k, b):
    """What is left at the last event of the first event's contribution.

    One pixel with events at t_0 = 0 and at the cumulative gaps after it;
    the state is linear in the polarities when nothing clamps, so half the
    difference between the runs with p_0 = +1 and p_0 = -1, over C, is the
    first event's residual."""
    t = np.concatenate([[0], np.cumsum(gaps_us)])
    out = []
    for p0 in (1, -1):
        ev = make_events([(int(ti), 0, 0, p0 if i == 0 else (1 if i % 2 else -1))
                          for i, ti in enumerate(t)])
        st = OracleState(1, 1, OracleParams(C=0.5, k_per_s=k, b=b, s_min=-BIG,
                                            s_max=BIG, method=method))
        st.integrate(ev)
        out.append(st.S[0])
    return (out[0] - out[1]) / (2 * 0.5)


@pytest.mark.parametrize("n", [2, 3, 8, 40])
@pytest.mark.parametrize("b", [0.7, 2.0])
def test_eq6_adaptivity_ab(n, b):
    # Eq. 6: n events spaced t apart leave d(t)^n of the first event's term
    # under ESI's decay (Alg. 1), more than the d(n t) a single gap leaves.
    # Eq. 3 with exp decay has no such rate dependence: exp(-k n t) either way.
    k, span = 10.0, 60_000                     # n t = 0.06 s < 1 / k
    dense = first_event_residual(1, [span // n] * n, k, b)
    sparse = first_event_residual(1, [span], k, b)
    assert dense == pytest.approx(d_np(span // n, k, b) ** n, rel=1e-12)
    assert sparse == pytest.approx(d_np(span, k, b), rel=1e-12)
    assert dense > sparse
    e_dense = first_event_residual(2, [span // n] * n, k, b)
    e_sparse = first_event_residual(2, [span], k, b)
    assert e_dense == pytest.approx(np.exp(-k * 1e-6 * span), rel=1e-12)
    assert e_sparse == pytest.approx(np.exp(-k * 1e-6 * span), rel=1e-12)


# -------------------------------------------------- Fig. 4 diagnostics
def fig4_levels():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fig4_noise_levels.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            thr, ratio, value = line.split()
            rows.append((float(thr), float(ratio), float(value)))
    return rows


@pytest.mark.parametrize("thr,ratio,value", fig4_levels())
def test_fig4_printed_noise_levels(thr, ratio, value):
    # the events that change the intensity by `ratio` at this threshold,
    # accumulated by Eq. 2 in event units (C = 1), map to the printed value
    n = int(round(np.log(ratio) / np.log(1.0 + thr)))
    for sign in (1, -1):
        st = OracleState(3, 2, OracleParams(C=1.0, k_per_s=0.0, b=1.0, s_min=-1.0,
                                            s_max=1.0, method=1))
        st.integrate(make_events([(10 * i, 2, 1, sign) for i in range(n)]))
        N = oracle.noise_map(st.S)
        assert round(float(N[1 * 3 + 2]), 1) == value
        assert np.all(N[np.arange(6) != 5] == 0.0)


def test_noise_map_of_eq2_accumulation():
    # ln(1 + C |n_plus - n_minus|) per pixel; zero where no net events, the
    # same for negated polarities
    rng = np.random.default_rng(50)
    W, H, C = 11, 9, 0.15
    ev = random_stream(rng, W, H, 6000, 2_000_000, pol_bias=0.6)
    p = OracleParams(C=C, k_per_s=0.0, b=1.0, s_min=-1.0, s_max=1.0, method=1)
    st = OracleState(W, H, p)
    st.integrate(ev)
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    net = np.bincount(pix, weights=np.where(ev["p"] > 0, 1, -1), minlength=W * H)
    np.testing.assert_allclose(oracle.noise_map(st.S), np.log1p(C * np.abs(net)),
                               rtol=1e-13, atol=1e-15)
    neg = ev.copy()
    neg["p"] = -neg["p"]
    st2 = OracleState(W, H, p)
    st2.integrate(neg)
    assert np.array_equal(oracle.noise_map(st2.S), oracle.noise_map(st.S))


def test_count_events_is_a_histogram():
    rng = np.random.default_rng(51)
    W, H = 13, 7
    ev = random_stream(rng, W + 3, H + 2, 9000, 10**6)     # some out of range
    inside = (ev["x"] < W) & (ev["y"] < H)
    pix = ev["y"][inside].astype(np.int64) * W + ev["x"][inside]
    expect = np.bincount(pix, minlength=W * H)
    assert np.array_equal(oracle.count_events(ev, W, H), expect)
    assert np.array_equal(oracle.count_events(ev[:0], W, H), np.zeros(W * H))


# ------------------------------------------------ continuous-time output
@pytest.mark.parametrize("method,b", [(1, 2.0), (1, 0.7), (2, 1.0)])
def test_event_states_are_eq5_prefixes(method, b):
    # S right after event j of a pixel is the clamp-free closed form over
    # that pixel's events up to j: the corrected Eq. 5 (methods 0/1) or
    # Eq. 3's sum (method 2); the last one is the final state
    rng = np.random.default_rng(80 + method)
    W, H, k, C = 5, 4, 8.0, 0.3
    ev = random_stream(rng, W + 1, H, 2500, 300_000)         # a column outside
    p = OracleParams(C=C, k_per_s=k, b=b, s_min=-0.2, s_max=0.2, method=method)
    st = OracleState(W, H, p)
    vals = st.event_states(ev)
    inside = ev["x"] < W
    assert np.all(np.isnan(vals[~inside])) and not np.any(np.isnan(vals[inside]))
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for q in range(W * H):
        sel = np.nonzero(inside & (pix == q))[0]
        if len(sel) == 0:
            continue
        t = ev["t"][sel]
        s = np.where(ev["p"][sel] > 0, 1.0, -1.0)
        for j in range(len(sel)):
            if method == 2:
                expect = C * np.sum(s[:j + 1] * np.exp(-k * 1e-6 * (t[j] - t[:j + 1])))
            else:
                tt = np.concatenate([[0], t[:j + 1]])
                expect = C * np.sum(s[:j + 1] * np.cumprod(d_np(np.diff(tt), k, b)[::-1])[::-1])
            assert vals[sel[j]] == pytest.approx(expect, rel=1e-11, abs=1e-15)
        assert vals[sel[-1]] == st.S[q]
    ref = OracleState(W, H, p)
    ref.integrate(ev)
    assert np.array_equal(ref.S, st.S) and np.array_equal(ref.T, st.T)


def test_event_states_with_clamp_stay_in_bounds_and_match_frames():
    # Alg. 2: each value is clamped; a frame with render_decay = 0 shows, per
    # pixel, the value after that pixel's last event up to the frame time
    rng = np.random.default_rng(85)
    W, H = 6, 5
    ev = random_stream(rng, W, H, 3000, 400_000, pol_bias=0.7)
    p = OracleParams(C=0.25, k_per_s=5.0, b=2.0, s_min=-0.5, s_max=0.75)
    vals = OracleState(W, H, p).event_states(ev)
    assert np.all((vals >= -0.5) & (vals <= 0.75))
    frames, _ = OracleState(W, H, p).replay(ev, [200_000])
    pix = ev["y"].astype(np.int64) * W + ev["x"]
    for q in range(W * H):
        sel = np.nonzero((pix == q) & (ev["t"] <= 200_000))[0]
        v = vals[sel[-1]] if len(sel) else 0.0
        assert frames[0].ravel()[q] == int(np.clip(np.rint(255 * (v + 0.5) / 1.25), 0, 255))
