"""Fig. 4 diagnostics on the CUDA path: the noise-accumulation map ln(1 + |S|)
and per-pixel event counts, against the oracle.

Map tolerance: the state carries the parity error of esi_harness (1e-5
relative, floor C), which ln(1 + |S|) shrinks by 1 / (1 + |S|); log1pf adds
a few ulp.  So |N_gpu - N_ref| <= 1e-5 max(|S_ref|, C) / (1 + |S_ref|)
+ 4e-7 N_ref.  Counts are integers: exact.
"""
import os

import numpy as np
import pytest

import oracle
from esi_harness import GpuStream, random_events, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def check_map(N_gpu, S_ref, C):
    N_ref = oracle.noise_map(S_ref)
    tol = 1e-5 * np.maximum(np.abs(S_ref), C) / (1.0 + np.abs(S_ref)) + 4e-7 * N_ref
    err = np.abs(N_gpu.astype(np.float64) - N_ref)
    assert np.all(err <= tol), float(np.max(err - tol))


EQ2_EVENTS = dict(C=1.0, k_per_s=0.0, b=1.0, s_min=-1.0, s_max=1.0, method=1)


@pytest.mark.parametrize("p", [
    EQ2_EVENTS,                                                   # Fig. 4 as drawn
    dict(C=0.15, k_per_s=0.0, b=1.0, s_min=-1.0, s_max=1.0, method=1),
    dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0),      # Alg. 2 state
    dict(C=0.2, k_per_s=20.0, b=1.0, s_min=-1.0, s_max=1.0, method=2),
])
@pytest.mark.parametrize("W,H", [(346, 260), (37, 19), (1, 1)])
def test_noise_map_matches_the_oracle(p, W, H):
    # 2 s of noise with two hot pixels, as in Fig. 4's recording
    import torch
    rng = np.random.default_rng(W * 3 + H + int(p["k_per_s"]))
    ev = random_events(rng, W, H, max(10, W * H // 2), 0, 2_000_000, hot=(W // 4, H // 2, 0.05))
    hot2 = ev["t"] % 7 == 0
    ev["x"][hot2], ev["y"][hot2] = W - 1, 0
    ref = run_oracle(ev, W, H, p, [2_000_000])
    with GpuStream(W, H, p) as g:
        g.esi.check(g.push(ev), "push")
        rc, _ = g.render_frames([2_000_000])
        g.esi.check(rc, "render")
        N = np.empty(W * H, dtype=np.float32)
        g.esi.check(g.esi.esi_noise_map(g.h, N, 0), "noise map (host)")
        check_map(N, ref["S"], p["C"])
        # device output, 16-byte aligned (vector path) and not (scalar path)
        buf = torch.empty(W * H + 1, dtype=torch.float32, device="cuda")
        for off in (0, 1):
            out = buf[off:off + W * H]
            g.esi.check(g.esi.esi_noise_map(g.h, out, 1), "noise map (device)")
            assert np.array_equal(out.cpu().numpy(), N)


def fig4_levels():
    path = os.path.join(os.path.dirname(__file__), "golden", "fig4_noise_levels.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            thr, ratio, value = line.split()
            rows.append((float(thr), float(ratio), float(value)))
    return rows


@pytest.mark.parametrize("thr,ratio,value", fig4_levels())
def test_fig4_printed_noise_levels_on_the_gpu(thr, ratio, value):
    from synth import EVENT_DTYPE
    n = int(round(np.log(ratio) / np.log(1.0 + thr)))
    W, H = 5, 3
    ev = np.zeros(2 * n, dtype=EVENT_DTYPE)
    ev["t"] = np.repeat(np.arange(n) * 10, 2)
    ev["x"] = np.tile([1, 4], n)
    ev["y"] = np.tile([2, 0], n)
    ev["p"] = np.tile([1, -1], n)
    with GpuStream(W, H, EQ2_EVENTS) as g:
        g.esi.check(g.push(ev), "push")
        g.esi.check(g.render_frames([10 * n])[0], "render")
        N = np.empty((H, W), dtype=np.float32)
        g.esi.check(g.esi.esi_noise_map(g.h, N, 0), "noise map")
    assert round(float(N[2, 1]), 1) == value and round(float(N[0, 4]), 1) == value
    N[2, 1] = N[0, 4] = 0.0
    assert np.all(N == 0.0)


@pytest.mark.parametrize("W,H,n", [(346, 260, 200_000), (37, 19, 5000), (3, 1, 0), (1280, 720, 20_000_000)])
def test_count_events_is_exact(W, H, n):
    import torch
    rng = np.random.default_rng(W + n)
    ev = random_events(rng, W + 2, H + 1, n, 0, 10**6, hot=(0, 0, 0.1))    # some outside
    expect = oracle.count_events(ev, W, H)
    p = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)
    with GpuStream(W, H, p) as g:
        c = np.full(W * H, 7, dtype=np.uint32)
        g.esi.check(g.esi.esi_count_events(g.h, ev, n, 0, c, 0), "count (host)")
        assert np.array_equal(c, expect)
        dev_ev = torch.from_numpy(ev.view(np.uint8).copy()).cuda()
        dc = torch.full((W * H,), 7, dtype=torch.int32, device="cuda")
        g.esi.check(g.esi.esi_count_events(g.h, dev_ev, n, 1, dc, 1), "count (device)")
        assert np.array_equal(dc.cpu().numpy().view(np.uint32), expect)
        # counting queues nothing: the handle's state and counters are untouched
        st = g.stats()
        assert st.events_pushed == 0 and st.frames_rendered == 0
