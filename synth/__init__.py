"""Seeded synthetic event streams (input fixtures for tests, oracle and bench).

This module holds no ESI arithmetic: it models an event camera (Sec. III-A,
Eq. 1) watching analytic scenes and returns time-ordered events.  Both the
oracle and the CUDA path consume its output; neither is imported here.

Event layout (16 bytes, little endian): int64 t (microseconds), uint16 x,
uint16 y, int8 p (polarity, >0 means +1), 3 padding bytes.

Workload recipes (seeds 1000, 1001, 1002):

* ``sinusoid_346x260`` 346x260, 1 s: sinusoid of 0.05 cycles/px translating at 200 px/s,
  C = 0.2 (2 % per-pixel mismatch), 0.1 Hz/px noise, amplitude tuned to
  about 1 M events.
* ``blobs_640x480`` 640x480, 2 s: 40 Gaussian blobs in log intensity (sigma 5-30 px,
  linear motion up to 1000 px/s, toroidal wrap), per-pixel C ~ N(0.15, 0.03),
  0.1 Hz/px noise, about 10 M events.
* ``checkerboard_1280x720`` 1280x720, 1 s: 32 px checkerboard rotating at 2 rad/s (log
  contrast 0.40, 1.5 px edges), two bursts (20 ms, 10 ms) of 100 Hz flicker of
  +-22 % intensity, 0.05 % hot pixels at 1-20 kHz (80 % positive), C = 0.2
  (3 % mismatch), about 50 M events with heavy-tailed per-pixel counts.
* ``serving_stream`` sinusoid form with a given seed, phase and event rate.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

EVENT_DTYPE = np.dtype([("t", "<i8"), ("x", "<u2"), ("y", "<u2"), ("p", "i1"),
                        ("pad", "u1", (3,))], align=False)
assert EVENT_DTYPE.itemsize == 16

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

MAX_BURSTS = 8


class Scene(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
        ("n_blobs", ctypes.c_int32),
        ("duration_s", ctypes.c_double), ("t0_us", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("C_mean", ctypes.c_double), ("C_rel_sigma", ctypes.c_double),
        ("noise_hz", ctypes.c_double),
        ("sin_mean", ctypes.c_double), ("sin_amp", ctypes.c_double),
        ("sin_freq_cpx", ctypes.c_double), ("sin_speed_pxs", ctypes.c_double),
        ("blob_sigma_min", ctypes.c_double), ("blob_sigma_max", ctypes.c_double),
        ("blob_speed_min", ctypes.c_double), ("blob_speed_max", ctypes.c_double),
        ("blob_amp_min", ctypes.c_double), ("blob_amp_max", ctypes.c_double),
        ("checker_px", ctypes.c_double), ("rot_rad_s", ctypes.c_double),
        ("checker_log_contrast", ctypes.c_double), ("edge_px", ctypes.c_double),
        ("flicker_hz", ctypes.c_double), ("flicker_log_depth", ctypes.c_double),
        ("flicker_ramp_s", ctypes.c_double),
        ("n_bursts", ctypes.c_int32), ("_pad0", ctypes.c_int32),
        ("burst_start_s", ctypes.c_double * MAX_BURSTS),
        ("burst_len_s", ctypes.c_double * MAX_BURSTS),
        ("hot_frac", ctypes.c_double), ("hot_rate_min", ctypes.c_double),
        ("hot_rate_max", ctypes.c_double), ("hot_pos_prob", ctypes.c_double),
        ("sin_phase_px", ctypes.c_double),
        ("keep_prob", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the generator (gcc, OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:],
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.syn_generate.argtypes = [ctypes.POINTER(Scene),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
            lib.syn_generate.restype = ctypes.c_void_p
            lib.syn_free.argtypes = [ctypes.c_void_p]
            lib.syn_free.restype = None
            lib.syn_copy.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            lib.syn_copy.restype = None
            _lib = lib
        return _lib


def generate(scene: Scene, out: np.ndarray | None = None, threads: int = 0) -> np.ndarray:
    """Run the sensor model; returns a structured array of EVENT_DTYPE.

    ``out`` may be a preallocated (e.g. pinned) uint8/EVENT_DTYPE buffer large
    enough for the result; a view of it is returned.
    """
    lib = _load()
    n = ctypes.c_int64(0)
    ptr = lib.syn_generate(ctypes.byref(scene), ctypes.byref(n), int(threads))
    try:
        count = int(n.value)
        if out is None:
            res = np.empty(count, dtype=EVENT_DTYPE)
        else:
            flat = out.view(np.uint8).reshape(-1)
            if flat.nbytes < count * 16:
                raise ValueError("output buffer too small")
            res = flat[: count * 16].view(EVENT_DTYPE)
        if count:
            lib.syn_copy(ptr, count, res.ctypes.data)
        return res
    finally:
        lib.syn_free(ptr)


def _base(kind: int, W: int, H: int, duration_s: float, seed: int, C: float,
          C_rel_sigma: float, noise_hz: float, t0_us: int = 0) -> Scene:
    s = Scene()
    s.kind, s.W, s.H = kind, W, H
    s.duration_s, s.t0_us, s.seed = duration_s, t0_us, seed
    s.C_mean, s.C_rel_sigma, s.noise_hz = C, C_rel_sigma, noise_hz
    return s


def sinusoid_amp_for_rate(rate_ev_s: float, W: int, H: int, C: float,
                          freq_cpx: float = 0.05, speed_pxs: float = 200.0,
                          mean: float = 0.5) -> float:
    """Largest row amplitude of the translating sinusoid for about rate_ev_s events/s.

    Row y has amplitude a (y + 0.5) / H.  Each period sweeps its log intensity
    over swing = ln((m + a_y) / (m - a_y)) and back, so a pixel fires about
    2 floor(swing / C) events per period; freq * speed periods pass per second.
    """
    periods = freq_cpx * speed_pxs

    def rate(a: float) -> float:
        tot = 0.0
        for y in range(H):
            ay = a * (y + 0.5) / H
            sw = math.log((mean + ay) / (mean - ay))
            tot += 2.0 * math.floor(sw / C) * periods
        return tot * W

    lo, hi = 0.0, mean * 0.999
    if rate(hi) < rate_ev_s:
        return hi
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if rate(mid) < rate_ev_s:
            lo = mid
        else:
            hi = mid
    return hi


# Measured (nominal, generated) events/s per pixel of the sinusoid scene
# (C = 0.2, 2 % mismatch, 0.05 cycles/px, 200 px/s); the nominal model above
# ignores that a row whose swing is under 2 C may never leave its reference.
_S0_CAL = np.array([
    (2.0e5, 6.736e4), (3.0e5, 1.1854e5), (4.5e5, 2.1749e5), (6.0e5, 3.3265e5),
    (8.0e5, 5.3351e5), (1.0e6, 7.0548e5), (1.3e6, 9.1894e5), (1.7e6, 1.3195e6),
    (2.2e6, 1.7168e6), (3.0e6, 2.4912e6), (4.0e6, 3.4462e6), (5.0e6, 4.4257e6),
    (6.5e6, 5.8550e6), (8.0e6, 7.3374e6)]) / (346.0 * 260.0)


def _s0_nominal(rate_ev_s: float, W: int, H: int) -> float:
    per_px = rate_ev_s / float(W * H)
    lx, ly = np.log(_S0_CAL[:, 1]), np.log(_S0_CAL[:, 0])
    return float(np.exp(np.interp(np.log(per_px), lx, ly,
                                  left=None, right=None))) * W * H


def sinusoid_346x260(duration_s: float = 1.0, seed: int = 1000, t0_us: int = 0,
            rate_ev_s: float = 1.0e6, W: int = 346, H: int = 260,
            phase_px: float = 0.0) -> Scene:
    s = _base(0, W, H, duration_s, seed, 0.2, 0.02, 0.1, t0_us)
    s.sin_mean, s.sin_freq_cpx, s.sin_speed_pxs = 0.5, 0.05, 200.0
    s.sin_amp = sinusoid_amp_for_rate(_s0_nominal(rate_ev_s, W, H), W, H, 0.2)
    s.sin_phase_px = phase_px
    return s


def blobs_640x480(duration_s: float = 2.0, seed: int = 1001, t0_us: int = 0,
            W: int = 640, H: int = 480, n_blobs: int = 40) -> Scene:
    s = _base(1, W, H, duration_s, seed, 0.15, 0.2, 0.1, t0_us)
    s.n_blobs = n_blobs
    s.blob_sigma_min, s.blob_sigma_max = 5.0, 30.0
    s.blob_speed_min, s.blob_speed_max = 100.0, 1000.0
    s.blob_amp_min, s.blob_amp_max = 0.4, 1.0
    return s


def checkerboard_1280x720(duration_s: float = 1.0, seed: int = 1002, t0_us: int = 0,
            W: int = 1280, H: int = 720) -> Scene:
    s = _base(2, W, H, duration_s, seed, 0.2, 0.03, 0.1, t0_us)
    s.checker_px, s.rot_rad_s, s.checker_log_contrast, s.edge_px = 32.0, 2.0, 0.40, 1.5
    s.flicker_hz, s.flicker_log_depth, s.flicker_ramp_s = 100.0, 0.45, 1e-3
    bursts = [(0.30, 0.02), (0.70, 0.01)]
    s.n_bursts = len(bursts)
    for i, (b0, bl) in enumerate(bursts):
        s.burst_start_s[i], s.burst_len_s[i] = b0, bl
    s.hot_frac, s.hot_rate_min, s.hot_rate_max, s.hot_pos_prob = 5e-4, 1e3, 2e4, 0.8
    return s


def serving_stream(index: int, rate_ev_s: float, duration_s: float,
                   W: int = 346, H: int = 260, base_seed: int = 1003,
                   t0_us: int = 0) -> Scene:
    """Sinusoid form stream number ``index`` (own seed and phase) at a target rate."""
    return sinusoid_346x260(duration_s=duration_s, seed=base_seed * 1000 + index,
                   t0_us=t0_us, rate_ev_s=rate_ev_s, W=W, H=H,
                   phase_px=(index * 7.3) % 20.0)


def lognormal_rates(n: int, seed: int, median: float = 1.0e6, sigma: float = 0.8,
                    lo: float = 0.2e6, hi: float = 5.0e6) -> np.ndarray:
    """Per-stream event rates, lognormal around ``median`` clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.clip(median * np.exp(sigma * rng.standard_normal(n)), lo, hi)


# Generated events/s of the blob and checkerboard scenes at their default sizes
# (over their first 0.25 s); thinning brings a stream of either form down to a
# lower target rate.
BLOBS_NATURAL_RATE = 4.9e6
CHECKER_NATURAL_RATE = 46.0e6
# the sinusoid calibration above reaches 8 Mev/s at 346x260
C0_MAX_RATE = 8.0e6


def mixed_serving(duration_s: float = 0.25, seed: int = 1004, counts=(16, 48, 128),
                  median: float = 1.0e6, sigma: float = 1.0, lo: float = 0.1e6,
                  hi: float = 20.0e6, late_join: float = 0.25, leave: float = 0.2,
                  scene_s: float | None = None):
    """Mixed-resolution serving workload: counts[0] 1280x720 checkerboard form,
    counts[1] 640x480 blob form and counts[2] 346x260 sinusoid form
    streams.  Rates are lognormal(median, sigma) clipped to [lo, hi] and to
    what each scene generates.  A fraction late_join of the streams joins at a
    seeded time in the first half (on a 1 ms grid), a fraction leave leaves at
    a seeded time in the second half.  Each stream's scene starts at its join
    time and ends at its leave time (or duration_s).

    scene_s: generate at most this much of each scene and repeat it in time
    (stream_events).

    Returns a list of dicts: form, W, H, rate, t_join_us, t_leave_us (None if
    it stays), t_end_us (its leave time or the end), scene.
    """
    rng = np.random.default_rng(seed)
    forms = [2] * counts[0] + [1] * counts[1] + [0] * counts[2]
    rates = np.clip(median * np.exp(sigma * rng.standard_normal(len(forms))), lo, hi)
    D = int(round(duration_s * 1e6))
    out = []
    for i, form in enumerate(forms):
        t_join = int(rng.integers(1, D // 2000)) * 1000 if rng.random() < late_join else 0
        t_leave = int(rng.integers(D // 2000, D // 1000)) * 1000 if rng.random() < leave else None
        dur = ((t_leave if t_leave is not None else D) - t_join) / 1e6
        if scene_s:
            dur = min(dur, scene_s)
        sd = seed * 1000 + i
        if form == 0:
            rate = float(min(rates[i], C0_MAX_RATE))
            sc = sinusoid_346x260(duration_s=dur, seed=sd, t0_us=t_join, rate_ev_s=rate,
                         phase_px=(i * 7.3) % 20.0)
        elif form == 1:
            rate = float(min(rates[i], BLOBS_NATURAL_RATE))
            sc = blobs_640x480(duration_s=dur, seed=sd, t0_us=t_join)
            sc.keep_prob = rate / BLOBS_NATURAL_RATE
        else:
            rate = float(min(rates[i], CHECKER_NATURAL_RATE))
            sc = checkerboard_1280x720(duration_s=dur, seed=sd, t0_us=t_join)
            sc.keep_prob = rate / CHECKER_NATURAL_RATE
        out.append(dict(form=form, W=sc.W, H=sc.H, rate=rate, t_join_us=t_join,
                        t_leave_us=t_leave, t_end_us=t_leave if t_leave is not None else D,
                        scene=sc))
    return out


def _arrivals(rng, t0_us: int, t1_us: int, mean_us: float = 1000.0) -> np.ndarray:
    """Packet arrival times in (t0, t1): Poisson with mean gap mean_us, plus a
    last one at t1 (the stream is complete up to each arrival)."""
    gaps = rng.exponential(mean_us, size=int((t1_us - t0_us) / mean_us) * 3 + 10)
    arr = t0_us + np.cumsum(gaps).astype(np.int64) + 1
    return np.append(arr[arr < t1_us], t1_us)


def serving_streams(n_streams: int = 64, duration_s: float = 0.25, seed: int = 1003,
                    scene_s: float | None = None):
    """Batched-serving workload of n_streams sinusoid form 346x260 streams:
    lognormal rates (median 1 Mev/s) clipped to [0.2, 5] Mev/s and Poisson
    packet arrivals with a 1 ms mean gap.  scene_s: generate at most this
    much of each stream's scene and repeat it in time (stream_events).

    Returns (rates, streams): each stream a dict with W, H, rate, scene,
    t_join_us, t_end_us and arrivals (int64 us; the last one at the end).
    """
    rates = lognormal_rates(n_streams, seed)
    rng = np.random.default_rng(seed)
    D = int(round(duration_s * 1e6))
    out = []
    for i in range(n_streams):
        sc = serving_stream(i, float(rates[i]), min(duration_s, scene_s or duration_s))
        out.append(dict(W=sc.W, H=sc.H, rate=float(rates[i]), scene=sc, t_join_us=0, t_end_us=D,
                        arrivals=_arrivals(rng, 0, D)))
    return rates, out


def stream_events(w: dict, t_end_us: int | None = None) -> np.ndarray:
    """A serving stream's events: its scene generated once and repeated in
    time (each copy shifted by the scene's length) up to its end time."""
    ev = generate(w["scene"])
    t0 = int(w.get("t_join_us", 0))
    t1 = int(t_end_us if t_end_us is not None else w["t_end_us"])
    period = int(round(w["scene"].duration_s * 1e6))
    if period <= 0 or t0 + period >= t1:
        return ev
    reps = -(-(t1 - t0) // period)
    out = np.concatenate([ev] * reps)
    out["t"] += np.repeat(np.arange(reps, dtype=np.int64) * period, len(ev))
    return out[out["t"] < t1]


def mixed_arrivals(ws, duration_s: float = 0.25, seed: int = 1004):
    """Poisson packet arrivals (1 ms mean gap) of every stream of a
    mixed_serving workload, from its join to its leave time (or the end)."""
    rng = np.random.default_rng(seed + 1)
    D = int(round(duration_s * 1e6))
    return [_arrivals(rng, w["t_join_us"], w["t_leave_us"] if w["t_leave_us"] is not None else D)
            for w in ws]


def pack_events(ev: np.ndarray, t_base_us: int) -> np.ndarray:
    """The 8-byte packed form of 16-byte events (the layout of esi.h's
    ESI_PACK_EVENT): x in bits 0..15, y in 16..31, polarity (p > 0) in bit
    32, t - t_base_us in bits 33..63.  Every time must lie in
    [t_base_us, t_base_us + 2^31)."""
    dt = ev["t"].astype(np.int64) - np.int64(t_base_us)
    if len(dt) and (dt.min() < 0 or dt.max() >= 2**31):
        raise ValueError("event times outside [t_base, t_base + 2^31)")
    w = ev["x"].astype(np.uint64)
    w |= ev["y"].astype(np.uint64) << np.uint64(16)
    w |= (ev["p"] > 0).astype(np.uint64) << np.uint64(32)
    w |= dt.astype(np.uint64) << np.uint64(33)
    return w
