"""The render's first sorting level, read back and checked bit for bit.

A render reorders each chunk of consecutive events by pixel tile before the
per-pixel update; pixels are independent (Eq. 5), so this is legal as long as
the sort is stable (Alg. 2 applies a pixel's events in stream order).  Here
the binning kernel runs alone through esi_bin_events on a device ring, and
every chunk's records and its column of the run table must equal what a
plain stable sort (numpy argsort, kind="stable") of the same events gives:
ties in time, hot pixels, events outside the sensor, a ring that wraps, both
ways the kernel finds same-tile lanes (mask words up to 1024 tiles, ballots
above), every tile row width.
"""
import numpy as np
import pytest

from esi_harness import random_events
from synth import EVENT_DTYPE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()


def expected(ev, W, H, tile_w, tile_h, chunk, t_base):
    """Per chunk: the records of its in-sensor events, stably sorted by tile,
    and per tile (start << 16 | count) within the chunk."""
    tiles_x = -(-W // tile_w)
    n_tiles = tiles_x * -(-H // tile_h)
    n = len(ev)
    n_chunks = -(-n // chunk)
    x = ev["x"].astype(np.int64)
    y = ev["y"].astype(np.int64)
    inside = (x < W) & (y < H)
    tile = (y // tile_h) * tiles_x + x // tile_w
    pit = (y % tile_h) * tile_w + x % tile_w
    pos = (ev["p"] > 0).astype(np.uint64)
    toff = (ev["t"] - t_base).astype(np.int64) & 0xffffffff
    rec = toff.astype(np.uint64) | (((pit.astype(np.uint64) << np.uint64(1)) | pos) << np.uint64(32))
    recs, runs = [], np.zeros((n_tiles, n_chunks), dtype=np.uint32)
    for c in range(n_chunks):
        sl = slice(c * chunk, min(n, (c + 1) * chunk))
        keep = inside[sl]
        tl = tile[sl][keep]
        order = np.argsort(tl, kind="stable")
        recs.append(rec[sl][keep][order])
        cnt = np.bincount(tl, minlength=n_tiles)
        start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        runs[:, c] = (start.astype(np.uint32) << np.uint32(16)) | cnt.astype(np.uint32)
    return recs, runs, int((~inside).sum())


def run_binning(ev, W, H, tile_w, tile_h, chunk, cap, first, t_base):
    import torch
    from paper_2508_02238_gb300 import esi
    n = len(ev)
    assert n <= cap
    ring = np.zeros(cap, dtype=EVENT_DTYPE)
    idx = (first + np.arange(n)) % cap
    ring[idx] = ev
    d_ring = torch.from_numpy(ring.view(np.uint8).copy()).cuda()
    n_chunks = -(-n // chunk)
    tiles_x = -(-W // tile_w)
    n_tiles = tiles_x * -(-H // tile_h)
    recs = torch.full((n_chunks * chunk,), -1, dtype=torch.int64, device="cuda")
    runs = torch.zeros((n_tiles, n_chunks), dtype=torch.int32, device="cuda")
    shape = esi.esi_tuning()
    shape.tile_w, shape.tile_h, shape.chunk_events = tile_w, tile_h, chunk
    rc, dropped = esi.esi_bin_events(W, H, shape, d_ring, cap, first, n, t_base, recs, runs)
    assert rc == 0, esi.esi_strerror(rc)
    return (recs.cpu().numpy().view(np.uint64), runs.cpu().numpy().view(np.uint32), dropped)


CASES = [
    # W, H, tile_w, tile_h, chunk: mask-word path (<= 1024 tiles) and ballot path
    (346, 260, 128, 8, 2048),
    (346, 260, 64, 8, 2048),
    (346, 260, 32, 32, 512),
    (640, 480, 128, 8, 4096),
    (1280, 720, 128, 8, 4096),
    (1280, 720, 64, 4, 1024),     # 3600 tiles: ballots over the tile index bits
    (1280, 720, 32, 16, 512),     # 1800 tiles
    (37, 19, 128, 4, 8192),
]


@pytest.mark.parametrize("W,H,tw,th,chunk", CASES)
def test_binning_is_a_stable_sort_by_tile(W, H, tw, th, chunk):
    rng = np.random.default_rng(W + 7 * H + tw + th + chunk)
    n = 3 * chunk + 777     # several chunks and a ragged tail
    ev = random_events(rng, W + 3, H + 2, n, 1000, 1000 + n // 2, hot=(W // 2, H // 3, 0.1))
    # ties: runs of equal time at one pixel with alternating polarity
    ev["x"][100:140], ev["y"][100:140] = 5 % W, 3 % H
    ev["t"][100:140] = ev["t"][100]
    ev["p"][100:140] = np.where(np.arange(40) % 2 == 0, 1, -1)
    ev["t"] = np.sort(ev["t"])
    cap = 1 << int(np.ceil(np.log2(n + 1)))
    first = cap - chunk // 2 - 5          # the ring wraps inside the second chunk
    t_base = int(ev["t"][0]) - 3
    recs, runs, dropped = run_binning(ev, W, H, tw, th, chunk, cap, first, t_base)
    want, want_runs, want_drop = expected(ev, W, H, tw, th, chunk, t_base)
    assert dropped == want_drop and want_drop > 0
    for c, r in enumerate(want):
        got = recs[c * chunk:c * chunk + len(r)]
        assert np.array_equal(got, r), f"chunk {c}: first mismatch at {np.argmax(got != r)}"
    assert np.array_equal(runs, want_runs)


def test_binning_of_a_scene_stream_with_wide_time_offsets():
    # a real scene's events (config-2 form, hot pixels), record times far from
    # t_base (the low 32 bits carry t - t_base exactly)
    import synth
    sc = synth.checkerboard_1280x720(duration_s=0.02)
    ev = synth.generate(sc)[:200_000]
    chunk = 4096
    cap = 1 << 18
    t_base = int(ev["t"][0]) - 3_000_000_000
    recs, runs, dropped = run_binning(ev, sc.W, sc.H, 128, 8, chunk, cap, 11, t_base)
    want, want_runs, want_drop = expected(ev, sc.W, sc.H, 128, 8, chunk, t_base)
    assert dropped == want_drop == 0
    for c, r in enumerate(want):
        assert np.array_equal(recs[c * chunk:c * chunk + len(r)], r), c
    assert np.array_equal(runs, want_runs)
