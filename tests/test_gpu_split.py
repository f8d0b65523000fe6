"""The split-row tile kernel (128-pixel rows).

A tile's rows are sorted as a whole into a scratch region and divided among
the tile's warps by work, a busy row split at record boundaries; the state at
a split comes from composing the row's earlier events as clamped-affine maps
(Alg. 2 with the clamp of Eq. 13; Alg. 1, Eq. 3 without).  With the splits
and the segmented scan off it must give the batch-walk kernel's results bit
for bit (same events, same order, same arithmetic); with splits on it must
match the FP64 oracle within the parity tolerance, on rows hot enough to be
split, for every method and render mode, tile height and launch shape,
including tiles with more records than one round of batches holds.
"""
import numpy as np
import pytest

from esi_harness import compare, random_events, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

BASE = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def hot_rows(seed, W, H, n, t1, rows=(3, 11), frac=0.4):
    """Random events plus hot pixels on a few rows, so that some tiles hold
    rows with several times their neighbours' records."""
    rng = np.random.default_rng(seed)
    ev = random_events(rng, W, H, n, 0, t1)
    sel = rng.random(n) < frac
    k = int(sel.sum())
    ev["y"][sel] = np.array(rows)[rng.integers(0, len(rows), size=k)] % H
    ev["x"][sel] = rng.integers(0, min(W, 40), size=k)
    ev["p"][sel] = np.where(rng.random(k) < 0.7, 1, -1)
    return ev


# 128-pixel rows: the split kernel's (small sensors default to 64-pixel rows)
SHAPES = [
    dict(tile_w=128, tile_h=8),
    dict(tile_w=128, tile_h=4),
    dict(tile_w=128, tile_h=16),
    dict(tile_w=128, tile_h=8, batch_records=1024, chunk_events=1024),     # several rounds of batches
    dict(tile_w=128, tile_h=8, max_batch_events=8192, chunk_events=1024),  # many sub-batches
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("W,H", [(256, 64), (301, 45)])
def test_sorted_rows_without_splits_equal_the_batch_walk(shape, W, H):
    ev = hot_rows(W + H + len(shape), W, H, 120_000, 600_000)
    p = dict(BASE, render_decay=1)
    tf = np.arange(7_000, 600_001, 7_000)
    walk = run_gpu(ev, W, H, p, tf, tuning={**shape, "scan_chain": 33, "split_rows": 2})
    rows = run_gpu(ev, W, H, p, tf, tuning={**shape, "scan_chain": 33, "split_rows": 3})
    compare(walk, run_oracle(ev, W, H, p, tf), p["C"], str(shape))
    for k in ("S", "T", "frames"):
        assert np.array_equal(walk[k], rows[k]), (k, shape)


METHODS = [
    dict(method=0, render_decay=1),
    dict(method=0, render_decay=0, b=1.7, k_per_s=40.0, s_min=-0.6, s_max=0.9),
    dict(method=1, render_decay=1, k_per_s=200.0),
    dict(method=2, render_decay=1, k_per_s=200.0),
    dict(method=0, render_decay=1, k_per_s=0.0, C=0.25, s_min=-2.0, s_max=2.0),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("over", METHODS)
def test_split_rows_match_the_oracle(shape, over):
    W, H = 256, 48
    ev = hot_rows(len(shape) * 13 + over["method"], W, H, 150_000, 500_000)
    p = dict(BASE, **over)
    tf = np.arange(9_000, 500_001, 9_000)
    for scan in (8, 33):
        got = run_gpu(ev, W, H, p, tf, tuning={**shape, "scan_chain": scan, "split_rows": 1})
        compare(got, run_oracle(ev, W, H, p, tf), p["C"], f"{shape} {over} scan {scan}")


def test_splits_happen_and_change_only_the_rounding():
    # a hot row next to quiet ones: the split kernel must split it (results
    # differ from the whole-row walk in the last bits) and stay within the
    # bar; the decay keeps a memory longer than a piece (k = 20 /s), so the
    # states at the splits come from composed maps that matter
    W, H = 128, 8
    rng = np.random.default_rng(5)
    ev = random_events(rng, W, H, 60_000, 0, 300_000)
    hot = rng.random(len(ev)) < 0.8
    ev["y"][hot] = 2
    p = dict(BASE, k_per_s=20.0, s_min=-40.0, s_max=40.0, render_decay=1)
    tf = np.arange(10_000, 300_001, 10_000)
    whole = run_gpu(ev, W, H, p, tf, tuning={"tile_w": 128, "scan_chain": 33, "split_rows": 3})
    split = run_gpu(ev, W, H, p, tf, tuning={"tile_w": 128, "scan_chain": 33, "split_rows": 1})
    ref = run_oracle(ev, W, H, p, tf)
    compare(whole, ref, p["C"], "whole rows")
    compare(split, ref, p["C"], "split rows")
    assert not np.array_equal(whole["S"], split["S"])
    assert np.array_equal(whole["T"], split["T"])


def test_split_rows_on_the_scene_streams():
    import synth
    sc = synth.checkerboard_1280x720(duration_s=0.12)
    ev = synth.generate(sc)
    p = dict(BASE, render_decay=1)
    for win in (10_000, 1_000):
        tf = np.arange(win, 120_001, win)
        compare(run_gpu(ev, sc.W, sc.H, p, tf), run_oracle(ev, sc.W, sc.H, p, tf), p["C"],
                f"checkerboard {win} us")


def test_split_rows_knob_validation():
    from esi_harness import GpuStream
    from paper_2508_02238_gb300 import esi
    with GpuStream(256, 32, dict(BASE)) as g:
        t = esi.esi_tuning()
        t.tile_w = 128
        for bad in (-1, 4):
            t.split_rows = bad
            assert esi.esi_set_tuning(g.h, t) == esi.ESI_EINVAL
        t.split_rows = 0
        assert esi.esi_set_tuning(g.h, t) == 0
        rc, got = esi.esi_get_tuning(g.h)
        assert rc == 0 and got.split_rows == 2
