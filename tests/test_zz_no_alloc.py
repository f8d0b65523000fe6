"""The allocation-free render entry point against the oracle and the handle path.

esi_render_frames_noalloc serves callers that cannot allocate device memory
(their application owns the GPU's memory in its own pool, or cudaMalloc's
device-wide synchronisation would stall a real-time loop); its scratch is a
fixed device array inside the library.  Two calls in a row, the second
continuing from the state the first left, must give what the FP64 oracle
gives and what esi_create / esi_push_events / esi_render_frames give for the
same events, within the parity tolerance of the other tests.  Inputs the call
must refuse (misaligned pointers, events out of time order, events after the
last frame or before their pixel's T, a time span beyond 32 bits) are made on
the host; each must return its error code and leave S, T and the frames as
they were.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from esi_harness import (GpuStream, compare, random_events, run_oracle, state_error,
                         STATE_TOL)
from synth import EVENT_DTYPE

pytestmark = pytest.mark.gpu

PARAMS = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, t_origin_us=0,
              render_decay=1)


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2508_02238_gb300 import esi
    esi.load_library()
    return torch, esi


def _dev_events(torch, ev, offset=0):
    """Device copy of the events starting `offset` bytes into a fresh buffer
    (offset 0: the allocation's own, 256-byte aligned start)."""
    raw = np.ascontiguousarray(ev, dtype=EVENT_DTYPE).view(np.uint8)
    buf = torch.zeros(len(raw) + 16 + offset, dtype=torch.uint8, device="cuda")
    buf[offset:offset + len(raw)] = torch.from_numpy(raw.copy()).cuda()
    return buf[offset:offset + len(raw)]


def _state(torch, P, t_origin, s_off=0, t_off=0):
    """S (zeros) and T (t_origin) as views `s_off` / `t_off` elements into
    their buffers, so an offset of one breaks their 16-byte alignment."""
    S = torch.zeros(P + s_off, dtype=torch.float32, device="cuda")[s_off:]
    T = torch.full((P + t_off,), t_origin, dtype=torch.int64, device="cuda")[t_off:]
    return S, T


def _two_calls(esi, torch, W, H, p, ev, cut, tfs, s_off=0, t_off=0):
    P = W * H
    prm = esi.make_params(**p)
    S, T = _state(torch, P, p["t_origin_us"], s_off, t_off)
    parts = [ev[ev["t"] <= cut], ev[ev["t"] > cut]]
    stream = torch.cuda.current_stream().cuda_stream
    frames_out = []
    for part, tf in zip(parts, tfs):
        dev_ev = _dev_events(torch, part)
        frames = torch.empty((len(tf), H, W), dtype=torch.uint8, device="cuda")
        rc = esi.esi_render_frames_noalloc(W, H, prm, dev_ev, len(part), tf, len(tf), S, T,
                                           frames, stream)
        assert rc == 0, esi.esi_strerror(rc)
        frames_out.append(frames.cpu().numpy())
    return frames_out, S.cpu().numpy(), T.cpu().numpy()


CASES = [
    # (W, H, render_decay, S offset, T offset): the vector path (W % 4 == 0,
    # 16-byte aligned state) and the scalar one (odd width, or state offset
    # by one element)
    (200, 120, 1, 0, 0),
    (346, 260, 1, 0, 0),
    (201, 120, 1, 0, 0),
    (200, 120, 0, 0, 0),
    (200, 120, 1, 1, 1),
]


@pytest.mark.parametrize("W,H,rd,s_off,t_off", CASES)
def test_noalloc_matches_oracle_and_handle_path_on_two_calls(W, H, rd, s_off, t_off):
    torch, esi = _setup()
    p = dict(PARAMS, render_decay=rd)
    rng = np.random.default_rng(W * 7 + H + rd)
    ev = random_events(rng, W, H, 200_000, 1, 1_000_000, hot=(7, 9, 0.02))
    cut = 500_000
    tfs = [np.arange(25_000, cut + 1, 25_000, dtype=np.int64),
           np.arange(cut + 25_000, 1_000_001, 25_000, dtype=np.int64)]
    got_frames, S, T = _two_calls(esi, torch, W, H, p, ev, cut, tfs, s_off, t_off)

    # the oracle, directly
    tf_all = np.concatenate(tfs)
    ref = run_oracle(ev, W, H, p, tf_all)
    compare({"S": S, "T": T, "frames": np.concatenate(got_frames)}, ref, p["C"],
            f"noalloc {W}x{H} rd={rd}")

    # the handle-based entry points on the same events
    parts = [ev[ev["t"] <= cut], ev[ev["t"] > cut]]
    with GpuStream(W, H, p) as g:
        for i, (part, tf) in enumerate(zip(parts, tfs)):
            assert g.push(part) == 0
            rc, fr = g.render_frames(tf)
            assert rc == 0
            assert np.abs(got_frames[i].astype(np.int16) - fr.astype(np.int16)).max() <= 1
        ref_S, ref_T = g.state()
    assert state_error(S, ref_S.astype(np.float64), p["C"]) <= STATE_TOL
    assert np.array_equal(T, ref_T)


def test_noalloc_with_no_events_renders_the_initial_state():
    torch, esi = _setup()
    W, H = 130, 40
    p = dict(PARAMS, t_origin_us=5_000)
    prm = esi.make_params(**p)
    S0 = np.linspace(-1.5, 1.5, W * H).astype(np.float32)
    T0 = np.full(W * H, 5_000, dtype=np.int64)
    S, T = torch.from_numpy(S0.copy()).cuda(), torch.from_numpy(T0.copy()).cuda()
    tf = np.array([5_000, 20_000, 60_000, 200_000], dtype=np.int64)
    frames = torch.empty((len(tf), H, W), dtype=torch.uint8, device="cuda")
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = esi.esi_render_frames_noalloc(W, H, prm, dummy, 0, tf, len(tf), S, T, frames, 0)
    assert rc == 0, esi.esi_strerror(rc)
    import oracle
    from esi_harness import oracle_params
    st = oracle.OracleState(W, H, oracle_params(p))
    st.S[:] = S0
    st.T[:] = T0
    ref = np.stack([st.render(int(t)) for t in tf])
    got = frames.cpu().numpy()
    assert np.abs(got.astype(np.int16) - ref.astype(np.int16)).max() <= 1
    assert np.array_equal(S.cpu().numpy(), S0) and np.array_equal(T.cpu().numpy(), T0)


def _refused(esi, torch, W, H, p, ev, tf, expect, ev_offset=0, S0=None, T0=None):
    """The call must return `expect` and leave S, T and frames untouched."""
    P = W * H
    S0 = np.zeros(P, dtype=np.float32) if S0 is None else S0
    T0 = np.full(P, p["t_origin_us"], dtype=np.int64) if T0 is None else T0
    S, T = torch.from_numpy(S0.copy()).cuda(), torch.from_numpy(T0.copy()).cuda()
    frames = torch.full((len(tf), H, W), 77, dtype=torch.uint8, device="cuda")
    dev_ev = _dev_events(torch, ev, ev_offset)
    rc = esi.esi_render_frames_noalloc(W, H, esi.make_params(**p), dev_ev, len(ev), tf, len(tf),
                                       S, T, frames, 0)
    assert rc == expect, (esi.esi_strerror(rc), esi.esi_strerror(expect))
    torch.cuda.synchronize()
    assert np.array_equal(S.cpu().numpy(), S0)
    assert np.array_equal(T.cpu().numpy(), T0)
    assert bool((frames == 77).all())


def test_noalloc_refuses_bad_inputs_and_leaves_the_state():
    torch, esi = _setup()
    W, H = 96, 40
    p = dict(PARAMS)
    rng = np.random.default_rng(11)
    ev = random_events(rng, W, H, 5_000, 10, 90_000)
    tf = np.array([50_000, 100_000], dtype=np.int64)
    # a device event buffer that is 8- but not 16-byte aligned: refused on the
    # host before any device access
    _refused(esi, torch, W, H, p, ev, tf, esi.ESI_EINVAL, ev_offset=8)
    # events out of time order
    bad = ev.copy()
    bad["t"][100], bad["t"][101] = bad["t"][101] + 5, bad["t"][100]
    _refused(esi, torch, W, H, p, bad, tf, esi.ESI_ETIMEORDER)
    # an event after the last frame
    late = ev.copy()
    late["t"][-1] = 100_001
    _refused(esi, torch, W, H, p, late, tf, esi.ESI_EINVAL)
    # an event earlier than its pixel's T
    T0 = np.full(W * H, p["t_origin_us"], dtype=np.int64)
    e0 = ev[0]
    T0[int(e0["y"]) * W + int(e0["x"])] = int(e0["t"]) + 1
    _refused(esi, torch, W, H, p, ev, tf, esi.ESI_ETIMEORDER, T0=T0)
    # a time span beyond 32 bits
    far = ev.copy()
    far["t"][-1] = far["t"][0] + (1 << 32)
    tf_far = np.array([50_000, int(far["t"][-1])], dtype=np.int64)
    _refused(esi, torch, W, H, p, far, tf_far, esi.ESI_ERANGE)
    # misaligned S (not 4-byte) or T (not 8-byte) pointers
    prm = esi.make_params(**p)
    S = torch.zeros(W * H + 4, dtype=torch.float32, device="cuda")
    T = torch.zeros(W * H + 2, dtype=torch.int64, device="cuda")
    frames = torch.empty((len(tf), H, W), dtype=torch.uint8, device="cuda")
    dev_ev = _dev_events(torch, ev)
    s_bad = S.view(torch.uint8)[2:2 + 4 * W * H]
    t_bad = T.view(torch.uint8)[4:4 + 8 * W * H]
    assert esi.esi_render_frames_noalloc(W, H, prm, dev_ev, len(ev), tf, len(tf), s_bad, T,
                                         frames, 0) == esi.ESI_EINVAL
    assert esi.esi_render_frames_noalloc(W, H, prm, dev_ev, len(ev), tf, len(tf), S, t_bad,
                                         frames, 0) == esi.ESI_EINVAL


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch, esi = _setup()
    p = esi.make_params(**PARAMS)
    W, H = 64, 32
    S = torch.zeros(W * H, dtype=torch.float32, device="cuda")
    T = torch.zeros(W * H, dtype=torch.int64, device="cuda")
    frames = torch.empty((1, H, W), dtype=torch.uint8, device="cuda")
    big = torch.zeros(16 * ((1 << 20) + 1), dtype=torch.uint8, device="cuda")
    tf = np.array([10], dtype=np.int64)
    assert esi.esi_render_frames_noalloc(W, H, p, big, (1 << 20) + 1, tf, 1, S, T, frames,
                                         0) == esi.ESI_ERANGE
    many = np.arange(1, 4098, dtype=np.int64)
    assert esi.esi_render_frames_noalloc(W, H, p, big, 0, many, len(many), S, T, frames,
                                         0) == esi.ESI_ERANGE
    assert esi.esi_render_frames_noalloc(4000, 4000, p, big, 0, tf, 1, S, T, frames,
                                         0) == esi.ESI_ERANGE
