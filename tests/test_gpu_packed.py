"""Packed 8-byte events (esi_push_packed) through the C ABI.

The words are built here from the bit layout esi.h states (x: bits 0-15,
y: 16-31, polarity: 32, time offset: 33-63), not by the library.  A packed
push must queue exactly the events an esi_push_events of the same events
queues: frames and state are compared bit for bit with a second handle fed
16-byte events, and once with the oracle.  Time-order violations (inside a
chunk, at a chunk boundary of the device check, against the previous push)
reject the whole push on every path."""
import numpy as np
import pytest

from esi_harness import GpuStream, compare, random_events, run_oracle

pytestmark = pytest.mark.gpu

W, H = 346, 260
PRM = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
CHUNK = 1 << 21          # events per device-checked chunk of a push
HOST_CHECK_MAX = 1 << 16  # host pushes up to this size are checked on the host


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def pack(ev, t_base):
    dt = ev["t"].astype(np.int64) - np.int64(t_base)
    assert dt.min() >= 0 and dt.max() < 2**31
    w = ev["x"].astype(np.uint64)
    w |= ev["y"].astype(np.uint64) << np.uint64(16)
    w |= (ev["p"] > 0).astype(np.uint64) << np.uint64(32)
    w |= dt.astype(np.uint64) << np.uint64(33)
    return w


def packets(seed, n, count, off_sensor=0):
    """count consecutive packets of n events, 100 ms each; off_sensor events
    per packet get x >= W (accepted and dropped)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        ev = random_events(rng, W, H, n, 1_000 + k * 100_000, 1_000 + (k + 1) * 100_000)
        if off_sensor:
            ev["x"][rng.integers(0, n, off_sensor)] = W + 3
        out.append(ev)
    return out


@pytest.mark.parametrize("n", [5_000, HOST_CHECK_MAX + 1, 2 * CHUNK + 12_345])
@pytest.mark.parametrize("on_device", [0, 1])
def test_packed_push_equals_event_push_bitwise(n, on_device):
    # three packets per handle: the ring (2^20 events at first) grows and wraps
    pk = packets(11 + n + on_device, n, 3, off_sensor=7)
    with GpuStream(W, H, PRM) as a, GpuStream(W, H, PRM) as b:
        for k, ev in enumerate(pk):
            t_base = int(ev["t"][0]) - 17
            assert a.push(ev, on_device=bool(on_device)) == 0
            assert b.push_packed(pack(ev, t_base), t_base, on_device=bool(on_device)) == 0
            tf = np.arange(1_000 + k * 100_000 + 25_000, 1_000 + (k + 1) * 100_000 + 1, 25_000)
            ra, fa = a.render_frames(tf)
            rb, fb = b.render_frames(tf)
            assert ra == 0 and rb == 0
            assert np.array_equal(fa, fb), k
        Sa, Ta = a.state()
        Sb, Tb = b.state()
        assert np.array_equal(Sa.view(np.uint32), Sb.view(np.uint32))
        assert np.array_equal(Ta, Tb)
        sa, sb = a.stats(), b.stats()
        assert sb.events_pushed == sa.events_pushed == 3 * n
        assert sb.events_dropped == sa.events_dropped == 21
        assert sb.last_event_t_us == sa.last_event_t_us == int(pk[-1]["t"][-1])


@pytest.mark.parametrize("on_device", [0, 1])
def test_packed_push_matches_the_oracle(on_device):
    rng = np.random.default_rng(5)
    ev = random_events(rng, W, H, 300_000, 0, 400_000, hot=(9, 4, 0.02))
    tf = np.arange(10_000, 400_001, 10_000)
    ref = run_oracle(ev, W, H, PRM, tf)
    with GpuStream(W, H, PRM) as g:
        assert g.push_packed(pack(ev, 0), 0, on_device=bool(on_device)) == 0
        rc, frames = g.render_frames(tf)
        assert rc == 0
        S, T = g.state()
        st = g.stats()
    compare({"S": S, "T": T, "frames": frames, "dropped": int(st.events_dropped)}, ref,
            PRM["C"], f"packed on_device={on_device}")


def _bad_orders(n):
    """(label, index) pairs: event index whose time goes below its predecessor's."""
    cases = [("inside", n // 3)]
    if n > CHUNK:
        cases.append(("chunk boundary", CHUNK))
    return cases


@pytest.mark.parametrize("n,on_device", [(4_000, 0), (CHUNK + 5_000, 0), (CHUNK + 5_000, 1),
                                         (4_000, 1)])
def test_packed_time_order_rejects_the_push(n, on_device):
    ev = packets(3, n, 1)[0]
    for label, i in _bad_orders(n):
        bad = ev.copy()
        bad["t"][i] = bad["t"][i - 1] - 1
        with GpuStream(W, H, PRM) as g:
            rc = g.push_packed(pack(bad, 0), 0, on_device=bool(on_device))
            assert rc == g.esi.ESI_ETIMEORDER, label
            assert g.stats().events_pushed == 0, label
            # the handle stays usable: the good push then renders as usual
            assert g.push_packed(pack(ev, 0), 0, on_device=bool(on_device)) == 0, label
            rc, fr = g.render_frames(np.array([int(ev["t"][-1])]))
            assert rc == 0 and g.stats().events_consumed == n, label
    # a push starting before the previous push's last event
    with GpuStream(W, H, PRM) as g:
        assert g.push_packed(pack(ev, 0), 0, on_device=bool(on_device)) == 0
        later = ev.copy()
        t_last = int(ev["t"][-1])
        later["t"] = t_last + 10 + np.arange(n)
        later["t"][0] = t_last - 1
        assert g.push_packed(pack(later, 0), 0, on_device=bool(on_device)) == g.esi.ESI_ETIMEORDER
        assert g.stats().events_pushed == n
        later["t"][0] = t_last       # equal times are in order
        assert g.push_packed(pack(later, 0), 0, on_device=bool(on_device)) == 0
        assert g.stats().last_event_t_us == int(later["t"][-1])


def test_packed_argument_checks():
    import torch
    ev = packets(4, 100, 1)[0]
    w = pack(ev, 0)
    with GpuStream(W, H, PRM) as g:
        esi = g.esi
        assert esi.esi_push_packed(g.h, None, 5, 0, 0) == esi.ESI_EINVAL
        assert esi.esi_push_packed(g.h, w, len(w), 0, 2) == esi.ESI_EINVAL
        assert esi.esi_push_packed(g.h, w, len(w), 2**62 + 1, 0) == esi.ESI_EINVAL
        assert esi.esi_push_packed(g.h, w, len(w), -(2**62) - 1, 0) == esi.ESI_EINVAL
        assert esi.esi_push_packed(g.h, w, 0, 0, 0) == esi.ESI_OK
        # a device array that is not 8-byte aligned is refused on the host
        buf = torch.zeros(len(w) * 8 + 8, dtype=torch.uint8, device="cuda")
        assert esi.esi_push_packed(g.h, buf[4:4 + len(w) * 8], len(w), 0, 1) == esi.ESI_EINVAL
        assert g.stats().events_pushed == 0
        # a time base far from zero: times are t_base + offset exactly
        t_base = 2**62 - 2**31
        w2 = pack(np.sort(ev.copy(), order="t"), 0)
        assert esi.esi_push_packed(g.h, w2, len(w2), t_base, 0) == esi.ESI_OK
        assert g.stats().last_event_t_us == t_base + int(ev["t"].max())
