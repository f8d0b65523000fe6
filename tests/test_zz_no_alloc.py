"""The allocation-free render entry point against the handle-based path.

esi_render_frames_noalloc serves callers that cannot allocate device memory
(their application owns the GPU's memory in its own pool, or cudaMalloc's
device-wide synchronisation would stall a real-time loop); its scratch is a
fixed device array inside the library.  Two calls in a row, the second
continuing from the state the first left, must give what esi_create /
esi_push_events / esi_render_frames give for the same events, within the
parity tolerance of the other tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from esi_harness import GpuStream, random_events, state_error, STATE_TOL

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


@pytest.mark.parametrize("W,H", [(200, 120), (346, 260)])
def test_noalloc_matches_handle_path_on_two_calls(W, H):
    torch, esi = _setup()
    rng = np.random.default_rng(W + H)
    ev = random_events(rng, W, H, 200_000, 1, 1_000_000, hot=(7, 9, 0.02))
    cut = 500_000
    parts = [ev[ev["t"] <= cut], ev[ev["t"] > cut]]
    tfs = [np.arange(25_000, cut + 1, 25_000, dtype=np.int64),
           np.arange(cut + 25_000, 1_000_001, 25_000, dtype=np.int64)]

    # reference: the handle-based entry points
    ref_frames = []
    with GpuStream(W, H, PARAMS) as g:
        for part, tf in zip(parts, tfs):
            assert g.push(part) == 0
            rc, fr = g.render_frames(tf)
            assert rc == 0
            ref_frames.append(fr)
        ref_S, ref_T = g.state()

    # the allocation-free call, twice in a row on caller-owned buffers
    P = W * H
    p = esi.make_params(**PARAMS)
    S = torch.zeros(P, dtype=torch.float32, device="cuda")
    T = torch.full((P,), PARAMS["t_origin_us"], dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for i, (part, tf) in enumerate(zip(parts, tfs)):
        dev_ev = torch.from_numpy(np.ascontiguousarray(part).view(np.uint8).copy()).cuda()
        frames = torch.empty((len(tf), H, W), dtype=torch.uint8, device="cuda")
        rc = esi.esi_render_frames_noalloc(W, H, p, dev_ev, len(part), tf, len(tf), S, T,
                                           frames, stream)
        assert rc == 0, esi.esi_strerror(rc)
        got = frames.cpu().numpy().astype(np.int16)
        assert np.abs(got - ref_frames[i].astype(np.int16)).max() <= 1
    S_h, T_h = S.cpu().numpy(), T.cpu().numpy()
    assert state_error(S_h, ref_S.astype(np.float64), PARAMS["C"]) <= STATE_TOL
    assert np.array_equal(T_h, ref_T)


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
