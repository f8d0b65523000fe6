"""The launch-shape autotuner (esi_autotune): its choice is a valid shape,
it leaves the handle's state and queued events alone, a cached choice is
reused, and the tuned handle still matches the FP64 oracle."""
import time

import numpy as np
import pytest

import synth
from esi_harness import GpuStream, compare, random_events, run_oracle

pytestmark = pytest.mark.gpu

P = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def _valid(t):
    return ((t.tile_w, t.tile_h) in {(128, 4), (128, 8), (128, 16), (64, 8), (64, 16), (32, 16),
                                     (32, 32)}
            and t.chunk_events in (2048, 4096) and t.batch_records in (2048, 4096)
            and t.max_batch_events in (1 << 21, 1 << 22, 1 << 23))


def test_autotune_keeps_state_and_matches_oracle():
    sc = synth.sinusoid_346x260()
    ev = synth.generate(sc)
    W, H = sc.W, sc.H
    tf = np.arange(10_000, 1_000_001, 10_000)
    half = np.searchsorted(ev["t"], 500_000)
    with GpuStream(W, H, P) as g:
        esi = g.esi
        esi.check(g.push(ev[:half]), "push")
        rc, f0 = g.render_frames(tf[:40])
        esi.check(rc, "render")
        # a sample later than anything queued: 0.1 s of the same scene
        sample = ev[np.searchsorted(ev["t"], 600_000):np.searchsorted(ev["t"], 700_000)].copy()
        stf = np.arange(610_000, 700_001, 10_000, dtype=np.int64)
        rc, chosen = esi.esi_autotune(g.h, sample, len(sample), stf, len(stf),
                                      esi.ESI_AUTOTUNE_FORCE)
        esi.check(rc, "esi_autotune")
        assert _valid(chosen)
        rc, cur = esi.esi_get_tuning(g.h)
        esi.check(rc, "esi_get_tuning")
        for f in ("tile_w", "tile_h", "chunk_events", "batch_records", "max_batch_events"):
            assert getattr(cur, f) == getattr(chosen, f), f
        # the handle goes on from where it was
        esi.check(g.push(ev[half:]), "push")
        rc, f1 = g.render_frames(tf[40:])
        esi.check(rc, "render")
        S, T = g.state()
    ref = run_oracle(ev, W, H, P, tf)
    gpu = {"S": S, "T": T, "frames": np.concatenate([f0, f1])}
    compare(gpu, ref, P["C"], "sinusoid 346x260 autotuned")


def test_autotune_cache_is_reused():
    rng = np.random.default_rng(11)
    W, H = 240, 180
    ev = random_events(rng, W, H, 200_000, 0, 200_000)
    tf = np.arange(10_000, 200_001, 10_000, dtype=np.int64)
    with GpuStream(W, H, P) as a, GpuStream(W, H, P) as b:
        esi = a.esi
        t0 = time.perf_counter()
        rc, first = esi.esi_autotune(a.h, ev, len(ev), tf, len(tf), esi.ESI_AUTOTUNE_FORCE)
        esi.check(rc, "autotune")
        measured = time.perf_counter() - t0
        t0 = time.perf_counter()
        rc, again = esi.esi_autotune(b.h, ev, len(ev), tf, len(tf), 0)
        esi.check(rc, "autotune cached")
        cached = time.perf_counter() - t0
        assert (again.tile_w, again.tile_h, again.chunk_events, again.batch_records,
                again.max_batch_events) == (first.tile_w, first.tile_h, first.chunk_events,
                                            first.batch_records, first.max_batch_events)
        assert cached < measured / 4, (cached, measured)
        rc, wide = esi.esi_autotune(a.h, ev, len(ev), tf, len(tf),
                                    esi.ESI_AUTOTUNE_FORCE | esi.ESI_AUTOTUNE_WIDE_ONLY)
        esi.check(rc, "autotune wide")
        assert wide.tile_w == 128 and _valid(wide)


def test_autotune_rejects_bad_samples():
    rng = np.random.default_rng(12)
    W, H = 64, 48
    ev = random_events(rng, W, H, 1000, 1000, 50_000)
    tf = np.array([20_000, 50_000], dtype=np.int64)
    with GpuStream(W, H, P) as g:
        esi = g.esi
        assert esi.esi_autotune(g.h, ev, 0, tf, 2)[0] == esi.ESI_EINVAL
        assert esi.esi_autotune(g.h, ev, len(ev), tf, 0)[0] == esi.ESI_EINVAL
        bad = ev.copy()
        bad["t"][10], bad["t"][11] = bad["t"][11] + 1, bad["t"][10]
        assert esi.esi_autotune(g.h, bad, len(bad), tf, 2)[0] == esi.ESI_ETIMEORDER
        assert esi.esi_autotune(g.h, ev, len(ev), tf[::-1].copy(), 2)[0] == esi.ESI_ETIMEORDER
