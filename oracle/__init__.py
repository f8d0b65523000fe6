"""FP64 CPU oracle for Event-based Single Integration (ESI).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it, and it imports nothing from the product.

The arithmetic lives in ``esi_oracle.c`` (plain C, IEEE double, no fused
multiply-add); this module only marshals numpy arrays.  It follows:

* Alg. 2 -- per event: S += p C; dt = t - T; S *= d(dt); T = t; clamp (Eq. 13).
* Eq. 4  -- d(t) = max(1 - k t, 0)^b (reading of max{(1-kt)^b, 0}).
* Eq. 14 -- B = 255 (S - S_min) / (S_max - S_min), round half to even,
  saturate; ``render_decay`` maps the view S d(t_frame - T) instead of S.
* ``method`` 1 -- Alg. 1: the same loop without the clamp (Eq. 2 when k = 0).
* ``method`` 2 -- Eq. 3 with d(t) = exp(-k t), no clamp, kept as the exact
  regrouping S <- S exp(-k (t - T)) + p C; T <- t of its sum.
* Fig. 4 -- the noise-accumulation map ln(1 + |S|); per-pixel event counts.
* Continuous-time output -- S of each event's pixel right after the event.

Pinned by ``tests/test_oracle_pins.py`` against closed forms the paper fixes
(Eq. 2, the corrected Eq. 5, Eq. 6), hand-worked cases, invariants and a
brute-force fold of the clamped-affine composition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

from synth import EVENT_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, IEEE semantics)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, d, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.oracle_decay.argtypes = [i64, d, d]
        lib.oracle_decay.restype = d
        lib.oracle_decay_exp.argtypes = [i64, d]
        lib.oracle_decay_exp.restype = d
        lib.oracle_init.argtypes = [P, P, i64, i64]
        lib.oracle_init.restype = None
        lib.oracle_integrate.argtypes = [P, i64, i32, i32, d, d, d, d, d, i32, P, P, P]
        lib.oracle_integrate.restype = i64
        lib.oracle_render.argtypes = [P, P, i64, d, d, d, d, i32, i32, i64, P]
        lib.oracle_render.restype = None
        lib.oracle_replay.argtypes = [P, i64, i32, i32, d, d, d, d, d, i32, i32,
                                      P, i64, P, P, P, P]
        lib.oracle_replay.restype = i64
        lib.oracle_event_states.argtypes = [P, i64, i32, i32, d, d, d, d, d, i32, P, P, P]
        lib.oracle_event_states.restype = None
        lib.oracle_noise_map.argtypes = [P, i64, P]
        lib.oracle_noise_map.restype = None
        lib.oracle_count_events.argtypes = [P, i64, i32, i32, P]
        lib.oracle_count_events.restype = None
        _lib = lib
        return lib


@dataclass(frozen=True)
class OracleParams:
    """ESI parameters: C (Alg. 2), k in 1/s and b (Eq. 4), clamp bounds (Eq. 13).

    method: 0 Alg. 2, 1 Alg. 1 (no clamp), 2 Eq. 3 with d(t) = exp(-k t).
    """
    C: float
    k_per_s: float
    b: float
    s_min: float
    s_max: float
    t_origin_us: int = 0
    render_decay: int = 0
    method: int = 0


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def decay(dt_us: int, k_per_s: float, b: float) -> float:
    """Eq. 4 (reading max(1 - k dt, 0)^b), dt in microseconds."""
    return float(_load().oracle_decay(int(dt_us), float(k_per_s), float(b)))


def decay_exp(dt_us: int, k_per_s: float) -> float:
    """The exponential decay exp(-k dt) used with Eq. 3, dt in microseconds."""
    return float(_load().oracle_decay_exp(int(dt_us), float(k_per_s)))


class OracleState:
    """S (float64) and T (int64 us) matrices of one W x H sensor, row-major."""

    def __init__(self, W: int, H: int, params: OracleParams):
        self.W, self.H, self.params = int(W), int(H), params
        P = self.W * self.H
        self.S = np.empty(P, dtype=np.float64)
        self.T = np.empty(P, dtype=np.int64)
        self.dropped = np.zeros(1, dtype=np.int64)
        _load().oracle_init(_ptr(self.S), _ptr(self.T), P, int(params.t_origin_us))

    def integrate(self, events: np.ndarray) -> int:
        """Apply events in push order (Alg. 2 loop).  Returns events applied."""
        ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
        p = self.params
        return int(_load().oracle_integrate(
            _ptr(ev), len(ev), self.W, self.H, p.C, p.k_per_s, p.b, p.s_min,
            p.s_max, int(p.method), _ptr(self.S), _ptr(self.T), _ptr(self.dropped)))

    def event_states(self, events: np.ndarray) -> np.ndarray:
        """Apply events in push order; S right after each (NaN if outside the sensor)."""
        ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
        out = np.empty(len(ev), dtype=np.float64)
        p = self.params
        _load().oracle_event_states(
            _ptr(ev), len(ev), self.W, self.H, p.C, p.k_per_s, p.b, p.s_min,
            p.s_max, int(p.method), _ptr(self.S), _ptr(self.T), _ptr(out))
        return out

    def render(self, t_frame_us: int, render_decay: int | None = None) -> np.ndarray:
        """Eq. 14 frame (uint8, H x W) at t_frame."""
        p = self.params
        rd = p.render_decay if render_decay is None else render_decay
        B = np.empty(self.W * self.H, dtype=np.uint8)
        _load().oracle_render(_ptr(self.S), _ptr(self.T), self.W * self.H,
                              p.k_per_s, p.b, p.s_min, p.s_max, int(rd),
                              int(p.method), int(t_frame_us), _ptr(B))
        return B.reshape(self.H, self.W)

    def replay(self, events: np.ndarray, t_frames) -> tuple[np.ndarray, int]:
        """Frames at each t_frames[w] after applying the events with t <= t_frames[w].

        Returns (frames[M, H, W] uint8, number of events consumed).
        """
        ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
        tf = np.ascontiguousarray(t_frames, dtype=np.int64)
        M = len(tf)
        B = np.empty((M, self.H, self.W), dtype=np.uint8)
        p = self.params
        used = _load().oracle_replay(
            _ptr(ev), len(ev), self.W, self.H, p.C, p.k_per_s, p.b, p.s_min,
            p.s_max, int(p.render_decay), int(p.method), _ptr(tf), M, _ptr(self.S),
            _ptr(self.T), _ptr(B), _ptr(self.dropped))
        return B, int(used)


def noise_map(S: np.ndarray) -> np.ndarray:
    """Fig. 4's map ln(1 + |S|) of a state (float64, same shape)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    N = np.empty_like(S)
    _load().oracle_noise_map(_ptr(S), S.size, _ptr(N))
    return N


def count_events(events: np.ndarray, W: int, H: int) -> np.ndarray:
    """Events per pixel (uint32, W * H row-major); out-of-range events skipped."""
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    counts = np.empty(int(W) * int(H), dtype=np.uint32)
    _load().oracle_count_events(_ptr(ev), len(ev), int(W), int(H), _ptr(counts))
    return counts
