"""Alg. 1 (no clamp) and Eq. 3 with exponential decay on the CUDA path.

Both run through the same kernels as Alg. 2 (esi_params.method); the oracle
runs each method's own loop.  Tolerances are those of esi_harness.
"""
import numpy as np
import pytest

from esi_harness import EXACT, compare, random_events, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ALG1, EQ3 = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def P(**kw):
    d = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-0.5, s_max=0.5)
    d.update(kw)
    return d


@pytest.mark.parametrize("W,H", [(100, 70), (346, 260), (37, 19)])
@pytest.mark.parametrize("method,b,k", [
    (ALG1, 2.0, 10.0), (ALG1, 1.3, 50.0), (ALG1, 3.0, 5.0), (ALG1, 2.0, 0.0),
    (EQ3, 2.0, 10.0), (EQ3, 2.0, 300.0), (EQ3, 2.0, 1e4), (EQ3, 2.0, 0.0),
])
@pytest.mark.parametrize("rd", [0, 1])
def test_methods_match_the_oracle(W, H, method, b, k, rd):
    # narrow bounds: Alg. 2 would clamp, these methods must not; the frames
    # saturate instead
    rng = np.random.default_rng(W + H + int(k) + 7 * method + rd)
    ev = random_events(rng, W, H, 30_000, 0, 500_000, hot=(W // 2, H // 3, 0.03))
    p = P(method=method, b=b, k_per_s=k, render_decay=rd)
    tf = np.arange(10_000, 500_001, 10_000)
    ref = run_oracle(ev, W, H, p, tf)
    got = run_gpu(ev, W, H, p, tf)
    compare(got, ref, p["C"], f"method {method} b={b} k={k} rd={rd}")
    if k > 0 and k < 1e3:
        assert np.max(np.abs(ref["S"])) > p["s_max"]     # unclamped state


TUNINGS = [
    dict(tile_h=4), dict(tile_h=16), dict(tile_w=32, tile_h=16), dict(tile_w=64, tile_h=8),
    dict(tile_w=32, tile_h=32, batch_records=1024, chunk_events=512),
    dict(max_batch_events=4096, chunk_events=512),
]


@pytest.mark.parametrize("method,b", [(ALG1, 2.0), (ALG1, 1.7), (EQ3, 2.0)])
def test_method_launch_shapes_bit_identical(method, b):
    rng = np.random.default_rng(60 + method)
    W, H = 200, 150
    ev = random_events(rng, W, H, 80_000, 0, 800_000, hot=(33, 40, 0.1))
    p = P(method=method, b=b, k_per_s=40.0, render_decay=1)
    tf = np.arange(10_000, 800_001, 10_000)
    ref = run_gpu(ev, W, H, p, tf, tuning=EXACT)
    compare(ref, run_oracle(ev, W, H, p, tf), p["C"])
    for t in TUNINGS:
        g = run_gpu(ev, W, H, p, tf, tuning={**t, **EXACT})
        assert np.array_equal(g["S"], ref["S"]), t
        assert np.array_equal(g["T"], ref["T"]), t
        assert np.array_equal(g["frames"], ref["frames"]), t


def test_eq3_k_zero_is_eq2_exactly():
    rng = np.random.default_rng(70)
    W, H = 70, 45
    ev = random_events(rng, W, H, 50_000, 0, 1_000_000)
    for method in (ALG1, EQ3):
        p = P(C=0.25, k_per_s=0.0, method=method)
        g = run_gpu(ev, W, H, p, [1_000_000])
        pix = ev["y"].astype(np.int64) * W + ev["x"]
        net = np.bincount(pix, weights=np.where(ev["p"] > 0, 1, -1), minlength=W * H)
        assert np.array_equal(g["S"].astype(np.float64), 0.25 * net)


def test_eq3_long_gaps_and_ties():
    # gaps beyond the FP32 range of exp(-k dt) (d = 0), gaps above 2^24 us,
    # and several events at one time (d = 1, order kept)
    W, H = 8, 4
    rows = []
    for x in range(W):
        for y in range(H):
            t = 0
            for j in range(6):
                t += [1, 0, 40_000_000, 3, 0, 123_457][j] * (1 + x)
                rows.append((t, x, y, 1 if (x + y + j) % 3 else -1))
    rows.sort(key=lambda r: r[0])
    from synth import EVENT_DTYPE
    ev = np.zeros(len(rows), dtype=EVENT_DTYPE)
    for i, (t, x, y, pol) in enumerate(rows):
        ev[i]["t"], ev[i]["x"], ev[i]["y"], ev[i]["p"] = t, x, y, pol
    t_end = int(ev["t"][-1])
    for k in (1.0, 10.0, 1e4):
        p = P(method=EQ3, k_per_s=k, render_decay=1)
        tf = [t_end // 3, t_end]
        compare(run_gpu(ev, W, H, p, tf), run_oracle(ev, W, H, p, tf), p["C"], f"k={k}")


def residual_maps(method, W, H, n_of_col, span, k, b):
    """The first event's residual at every pixel, measured on the GPU.

    Pixel (x, y) gets a marker event at t = 0 and n_of_col[x] more events
    evenly spaced up to about `span`, with alternating polarity.  Nothing
    clamps, so the state is linear in the polarities: half the difference
    of the runs with marker polarity +1 and -1, over C, is what is left of
    the marker's term."""
    from synth import EVENT_DTYPE
    C = 0.2
    rows = []
    for x in range(W):
        n = int(n_of_col[x])
        gap = span // n
        for y in range(H):
            rows.append((0, x, y, 0))
            for j in range(1, n + 1):
                rows.append((j * gap, x, y, 1 if j % 2 else -1))
    rows.sort(key=lambda r: r[0])
    ev = np.zeros(len(rows), dtype=EVENT_DTYPE)
    for i, (t, x, y, pol) in enumerate(rows):
        ev[i]["t"], ev[i]["x"], ev[i]["y"], ev[i]["p"] = t, x, y, pol
    marker = ev["t"] == 0
    out = []
    for sign in (1, -1):
        e = ev.copy()
        e["p"][marker] = sign
        p = P(C=C, k_per_s=k, b=b, method=method)
        g = run_gpu(e, W, H, p, [span + 1])
        compare(g, run_oracle(e, W, H, p, [span + 1]), C, f"method {method} marker {sign}")
        out.append(g["S"].astype(np.float64))
    s_plus, s_minus = out
    return ((s_plus - s_minus) / (2 * C)).reshape(H, W)


def test_eq6_adaptivity_ab_on_the_gpu():
    # Eq. 6 on a synthetic rate ramp: the more events a pixel sees over the
    # same span, the more of an old event ESI keeps (d(t)^n > d(n t));
    # Eq. 3 with exponential decay keeps exp(-k span) at any rate
    W, H, span, k, b = 40, 8, 80_000, 10.0, 2.0
    n_of_col = np.arange(1, W + 1)
    esi = residual_maps(ALG1, W, H, n_of_col, span, k, b)
    eq3 = residual_maps(EQ3, W, H, n_of_col, span, k, b)
    gaps = span // n_of_col
    u = 1.0 - k * 1e-6 * gaps
    expect_esi = (u ** b) ** n_of_col
    expect_eq3 = np.exp(-k * 1e-6 * gaps * n_of_col)
    for y in range(H):
        np.testing.assert_allclose(esi[y], expect_esi, rtol=2e-5)
        np.testing.assert_allclose(eq3[y], expect_eq3, rtol=2e-5)
    # same total span (to within a gap's rounding): ESI's residual grows with
    # the event rate, Eq. 3's does not
    exact = (span % n_of_col) == 0
    assert np.all(np.diff(esi[0][exact]) > 0)
    assert np.ptp(eq3[0][exact]) < 1e-5
