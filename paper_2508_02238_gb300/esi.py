"""ctypes binding of libesi.so: the C ABI of include/esi.h, same names.

Argument marshalling only.  Every step of the hot path runs in the CUDA
kernels of libesi.so; if the library cannot be built or loaded this module
raises instead of falling back to anything else.  Pointers may be given as
ints, numpy arrays (host memory) or torch tensors (``data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ESI_OK = 0
ESI_EINVAL = -1
ESI_ENOMEM = -2
ESI_EBUSY = -3
ESI_ETIMEORDER = -4
ESI_ERANGE = -5
ESI_ECUDA = -6
ESI_ETIMEOUT = -7
ESI_ESTATE = -8

# esi_params.method
ESI_METHOD_ALG2, ESI_METHOD_ALG1, ESI_METHOD_EQ3_EXP = 0, 1, 2
ESI_PACK_T_SHIFT = 33   # packed events: time offset in bits 33..63


class esi_params(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double), ("k_per_s", ctypes.c_double),
                ("b", ctypes.c_double), ("s_min", ctypes.c_double),
                ("s_max", ctypes.c_double), ("t_origin_us", ctypes.c_int64),
                ("render_decay", ctypes.c_int32), ("method", ctypes.c_int32)]


class esi_stats(ctypes.Structure):
    _fields_ = [("events_pushed", ctypes.c_uint64), ("events_consumed", ctypes.c_uint64),
                ("events_dropped", ctypes.c_uint64), ("events_pending", ctypes.c_uint64),
                ("frames_rendered", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("last_event_t_us", ctypes.c_int64), ("last_frame_t_us", ctypes.c_int64),
                ("ring_capacity", ctypes.c_uint64), ("ring_grows", ctypes.c_uint64),
                ("push_waits", ctypes.c_uint64)]


class esi_tuning(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("chunk_events", ctypes.c_int32),
                ("batch_records", ctypes.c_int32), ("max_batch_events", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("scan_chain", ctypes.c_int32),
                ("split_rows", ctypes.c_int32)]


class esi_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class esi_server_opts(ctypes.Structure):
    _fields_ = [("frame_period_us", ctypes.c_int64), ("max_events_per_tick", ctypes.c_int64),
                ("max_streams", ctypes.c_int32), ("frame_slots", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("max_stream_pixels", ctypes.c_int32), ("scan_chain", ctypes.c_int32),
                ("apply_mode", ctypes.c_int32), ("copy_threads", ctypes.c_int32),
                ("fuse_tick", ctypes.c_int32), ("_reserved", ctypes.c_int32),
                ("host_pool_bytes", ctypes.c_int64)]


class esi_server_stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_uint64), ("frames", ctypes.c_uint64),
                ("events", ctypes.c_uint64), ("packets", ctypes.c_uint64),
                ("frame_latency_p50_ms", ctypes.c_double), ("frame_latency_p99_ms", ctypes.c_double),
                ("packet_latency_p50_ms", ctypes.c_double), ("packet_latency_p99_ms", ctypes.c_double),
                ("gpu_ms_per_tick", ctypes.c_double), ("state_bytes_used", ctypes.c_uint64),
                ("state_budget_bytes", ctypes.c_uint64), ("streams_open", ctypes.c_int32),
                ("kernel_launches_per_tick", ctypes.c_int32),
                ("streams_admitted", ctypes.c_uint64), ("streams_refused", ctypes.c_uint64),
                ("events_refused", ctypes.c_uint64), ("host_tick_p50_ms", ctypes.c_double),
                ("host_tick_p99_ms", ctypes.c_double), ("gpu_tick_p99_ms", ctypes.c_double),
                ("host_pool_bytes", ctypes.c_uint64), ("host_pool_used_bytes", ctypes.c_uint64),
                ("host_pool_peak_bytes", ctypes.c_uint64), ("ring_grows", ctypes.c_uint64),
                ("events_dropped", ctypes.c_uint64)]


ESI_PACKET_EVENTS, ESI_PACKET_OPEN, ESI_PACKET_CLOSE = 0, 1, 2
ESI_APPLY_EVERY_TICK, ESI_APPLY_AT_FRAMES = 1, 2


class esi_tick_trace(ctypes.Structure):
    _fields_ = [("call_ns", ctypes.c_int64), ("issued_ns", ctypes.c_int64),
                ("ready_ns", ctypes.c_int64), ("copy_ms", ctypes.c_float),
                ("kernels_ms", ctypes.c_float), ("gap_ms", ctypes.c_float),
                ("frames", ctypes.c_int32), ("events", ctypes.c_int64),
                ("streams", ctypes.c_int32), ("items", ctypes.c_int32)]


class esi_packet(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("arrival_us", ctypes.c_int64), ("ev", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class esi_stream_spec(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("stream_id", ctypes.c_int32), ("params", esi_params),
                ("frame_sink", ctypes.c_void_p), ("sink_frames", ctypes.c_uint64),
                ("sink_t_frames", ctypes.c_void_p)]


_P = ctypes.c_void_p
_i32, _i64, _sz = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t

# name -> (restype, argtypes); the declarations of include/esi.h
SIGNATURES = {
    "esi_create": (_i32, [_i32, _i32, ctypes.POINTER(esi_params), _P, ctypes.POINTER(_P)]),
    "esi_push_events": (_i32, [_P, _P, _sz, _i32]),
    "esi_push_packed": (_i32, [_P, _P, _sz, _i64, _i32]),
    "esi_render_frame": (_i32, [_P, _i64, _P, _i32]),
    "esi_render_frames": (_i32, [_P, _P, _sz, _P, _i32]),
    "esi_get_state": (_i32, [_P, _P, _P, _i32]),
    "esi_set_state": (_i32, [_P, _P, _P, _i32]),
    "esi_synchronize": (_i32, [_P]),
    "esi_noise_map": (_i32, [_P, _P, _i32]),
    "esi_event_states": (_i32, [_P, _P, ctypes.c_size_t, _i32, ctypes.POINTER(ctypes.c_size_t)]),
    "esi_count_events": (_i32, [_P, _P, ctypes.c_size_t, _i32, _P, _i32]),
    "esi_get_stats": (_i32, [_P, ctypes.POINTER(esi_stats)]),
    "esi_set_tuning": (_i32, [_P, ctypes.POINTER(esi_tuning)]),
    "esi_get_tuning": (_i32, [_P, ctypes.POINTER(esi_tuning)]),
    "esi_autotune": (_i32, [_P, _P, _sz, _P, _sz, _i32, ctypes.POINTER(esi_tuning)]),
    "esi_profile_enable": (_i32, [_P, _i32]),
    "esi_profile_read": (_i32, [_P, ctypes.POINTER(esi_kernel_time), _i32]),
    "esi_profile_reset": (_i32, [_P]),
    "esi_destroy": (None, [_P]),
    "esi_strerror": (ctypes.c_char_p, [_i32]),
    "esi_render_frames_noalloc": (_i32, [_i32, _i32, ctypes.POINTER(esi_params), _P, _sz, _P,
                                         _sz, _P, _P, _P, _P]),
    "esi_server_create": (_i32, [_sz, ctypes.POINTER(esi_server_opts), _P, ctypes.POINTER(_P)]),
    "esi_stream_open": (_i32, [_P, _i32, _i32, ctypes.POINTER(esi_params), ctypes.POINTER(_i32)]),
    "esi_stream_push": (_i32, [_P, _i32, _P, _sz]),
    "esi_server_tick": (_i32, [_P, _i64]),
    "esi_server_trace": (_i32, [_P, _P, _sz, ctypes.POINTER(_sz)]),
    "esi_server_last_error": (ctypes.c_char_p, [_P]),
    "esi_stream_watermark": (_i32, [_P, _i32, _i64]),
    "esi_stream_set_tile_h": (_i32, [_P, _i32, _i32]),
    "esi_stream_autotune": (_i32, [_P, _i32, _P, _sz, _i32, ctypes.POINTER(_i32)]),
    "esi_server_run": (_i32, [_P, _P, _sz, _i64, _i64, _i32]),
    "esi_plain_run": (_i32, [_i32, _P, _P, _P, _P, _sz, _i64, _i64, _i64, _i32,
                             ctypes.POINTER(esi_server_stats)]),
    "esi_stream_frame": (_i32, [_P, _i32, _P, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)]),
    "esi_stream_frames_done": (_i32, [_P, _i32, ctypes.POINTER(ctypes.c_uint64)]),
    "esi_stream_set_frame_sink": (_i32, [_P, _i32, _P, ctypes.c_uint64, _P]),
    "esi_stream_frame_seq": (_i32, [_P, _i32, ctypes.c_uint64, _P, ctypes.POINTER(_i64)]),
    "esi_bin_events": (_i32, [_i32, _i32, ctypes.POINTER(esi_tuning), _P, ctypes.c_uint64,
                              ctypes.c_uint64, _sz, _i64, _P, _P,
                              ctypes.POINTER(ctypes.c_uint64), _P]),
    "esi_stream_state": (_i32, [_P, _i32, _P, _P]),
    "esi_stream_close": (_i32, [_P, _i32]),
    "esi_server_sync": (_i32, [_P]),
    "esi_server_get_stats": (_i32, [_P, ctypes.POINTER(esi_server_stats)]),
    "esi_server_reset_stats": (_i32, [_P]),
    "esi_server_destroy": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libesi.so (building it first if needed); raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libesi.so is not built; run paper_2508_02238_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def ptr(x) -> int:
    """Address of an int, a numpy array or a torch tensor (0 for None)."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _fn(name):
    return getattr(load_library(), name)


def esi_strerror(code: int) -> str:
    return _fn("esi_strerror")(int(code)).decode()


def esi_create(width: int, height: int, params: esi_params, cuda_stream=0):
    """Returns (rc, handle)."""
    h = _P()
    rc = _fn("esi_create")(int(width), int(height), ctypes.byref(params),
                           _P(int(cuda_stream) or None), ctypes.byref(h))
    return rc, h


def esi_push_events(h, ev, n: int, ev_on_device: int) -> int:
    return _fn("esi_push_events")(h, _P(ptr(ev) or None), int(n), int(ev_on_device))


def esi_push_packed(h, pk, n: int, t_base_us: int, pk_on_device: int) -> int:
    return _fn("esi_push_packed")(h, _P(ptr(pk) or None), int(n), int(t_base_us),
                                  int(pk_on_device))


def esi_render_frame(h, t_frame_us: int, out, out_on_device: int) -> int:
    return _fn("esi_render_frame")(h, int(t_frame_us), _P(ptr(out) or None), int(out_on_device))


def esi_render_frames(h, t_frames, m: int, out, out_on_device: int) -> int:
    return _fn("esi_render_frames")(h, _P(ptr(t_frames) or None), int(m),
                                    _P(ptr(out) or None), int(out_on_device))


def esi_get_state(h, S, T, on_device: int) -> int:
    return _fn("esi_get_state")(h, _P(ptr(S) or None), _P(ptr(T) or None), int(on_device))


def esi_set_state(h, S, T, on_device: int) -> int:
    return _fn("esi_set_state")(h, _P(ptr(S) or None), _P(ptr(T) or None), int(on_device))


def esi_synchronize(h) -> int:
    return _fn("esi_synchronize")(h)


def esi_event_states(h, out, cap: int, on_device: int):
    """Returns (rc, number of events applied)."""
    n = ctypes.c_size_t(0)
    rc = _fn("esi_event_states")(h, _P(ptr(out) or None), int(cap), int(on_device), ctypes.byref(n))
    return rc, int(n.value)


def esi_noise_map(h, out, on_device: int) -> int:
    return _fn("esi_noise_map")(h, _P(ptr(out) or None), int(on_device))


def esi_count_events(h, events, n: int, events_on_device: int, counts, counts_on_device: int) -> int:
    return _fn("esi_count_events")(h, _P(ptr(events) or None), int(n), int(events_on_device),
                                   _P(ptr(counts) or None), int(counts_on_device))


def esi_get_stats(h):
    st = esi_stats()
    rc = _fn("esi_get_stats")(h, ctypes.byref(st))
    return rc, st


def esi_set_tuning(h, t: esi_tuning) -> int:
    return _fn("esi_set_tuning")(h, ctypes.byref(t))


def esi_get_tuning(h):
    t = esi_tuning()
    rc = _fn("esi_get_tuning")(h, ctypes.byref(t))
    return rc, t


ESI_AUTOTUNE_FORCE = 1
ESI_AUTOTUNE_WIDE_ONLY = 2


def esi_autotune(h, sample, n: int, t_frames, m: int, flags: int = 0):
    """Returns (rc, chosen esi_tuning)."""
    t = esi_tuning()
    rc = _fn("esi_autotune")(h, _P(ptr(sample) or None), int(n), _P(ptr(t_frames) or None),
                             int(m), int(flags), ctypes.byref(t))
    return rc, t


def esi_profile_enable(h, enable: int) -> int:
    return _fn("esi_profile_enable")(h, int(enable))


def esi_profile_read(h, max_entries: int = 16):
    arr = (esi_kernel_time * max_entries)()
    n = _fn("esi_profile_read")(h, arr, int(max_entries))
    if n < 0:
        return n, {}
    return ESI_OK, {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
                    for i in range(min(n, max_entries))}


def esi_profile_reset(h) -> int:
    return _fn("esi_profile_reset")(h)


def esi_render_frames_noalloc(width: int, height: int, params: esi_params, events, n: int,
                              t_frames, m: int, S, T, frames, cuda_stream=0) -> int:
    return _fn("esi_render_frames_noalloc")(
        int(width), int(height), ctypes.byref(params), _P(ptr(events) or None), int(n),
        _P(ptr(t_frames) or None), int(m), _P(ptr(S) or None), _P(ptr(T) or None),
        _P(ptr(frames) or None), _P(int(cuda_stream) or None))


def esi_destroy(h) -> None:
    _fn("esi_destroy")(h)


def esi_server_create(state_budget_bytes: int, opts: esi_server_opts | None = None, cuda_stream=0):
    """Returns (rc, server)."""
    srv = _P()
    rc = _fn("esi_server_create")(int(state_budget_bytes),
                                  ctypes.byref(opts) if opts is not None else None,
                                  _P(int(cuda_stream) or None), ctypes.byref(srv))
    return rc, srv


def esi_stream_open(srv, width: int, height: int, params: esi_params):
    """Returns (rc, stream_id)."""
    sid = ctypes.c_int32(-1)
    rc = _fn("esi_stream_open")(srv, int(width), int(height), ctypes.byref(params), ctypes.byref(sid))
    return rc, int(sid.value)


def esi_stream_push(srv, stream_id: int, ev, n: int) -> int:
    return _fn("esi_stream_push")(srv, int(stream_id), _P(ptr(ev) or None), int(n))


def esi_server_tick(srv, now_us: int) -> int:
    return _fn("esi_server_tick")(srv, int(now_us))


def esi_stream_watermark(srv, stream_id: int, t_us: int) -> int:
    return _fn("esi_stream_watermark")(srv, int(stream_id), int(t_us))


def esi_stream_set_tile_h(srv, stream_id: int, tile_h: int) -> int:
    return _fn("esi_stream_set_tile_h")(srv, int(stream_id), int(tile_h))


def esi_stream_autotune(srv, stream_id: int, sample, n: int, flags: int = 0):
    """Returns (rc, chosen tile height)."""
    th = _i32(0)
    rc = _fn("esi_stream_autotune")(srv, int(stream_id), _P(ptr(sample) or None), int(n),
                                    int(flags), ctypes.byref(th))
    return rc, int(th.value)


def esi_server_run(srv, packets, n: int, tick_us: int, t_end_us: int, realtime: int) -> int:
    """packets: a ctypes array of esi_packet sorted by arrival_us."""
    return _fn("esi_server_run")(srv, ctypes.cast(packets, _P), int(n), int(tick_us),
                                 int(t_end_us), int(realtime))


def esi_plain_run(widths, heights, params, packets, n: int, tick_us: int, t_end_us: int,
                  frame_period_us: int, realtime: int):
    """widths, heights: int lists; params: list of esi_params.  Returns (rc, stats)."""
    ns = len(widths)
    W = (ctypes.c_int * ns)(*widths)
    H = (ctypes.c_int * ns)(*heights)
    Pm = (esi_params * ns)(*params)
    st = esi_server_stats()
    rc = _fn("esi_plain_run")(ns, ctypes.cast(W, _P), ctypes.cast(H, _P), ctypes.cast(Pm, _P),
                              ctypes.cast(packets, _P), int(n), int(tick_us), int(t_end_us),
                              int(frame_period_us), int(realtime), ctypes.byref(st))
    return rc, st


def esi_stream_frame(srv, stream_id: int, out):
    """Returns (rc, t_frame_us, latency_ms)."""
    t = ctypes.c_int64(0)
    lat = ctypes.c_double(0.0)
    rc = _fn("esi_stream_frame")(srv, int(stream_id), _P(ptr(out) or None), ctypes.byref(t),
                                 ctypes.byref(lat))
    return rc, int(t.value), float(lat.value)


def esi_stream_frames_done(srv, stream_id: int):
    """Returns (rc, number of the stream's finished frames)."""
    n = ctypes.c_uint64(0)
    rc = _fn("esi_stream_frames_done")(srv, int(stream_id), ctypes.byref(n))
    return rc, int(n.value)


def esi_stream_set_frame_sink(srv, stream_id: int, out, max_frames: int, t_frames=None) -> int:
    return _fn("esi_stream_set_frame_sink")(srv, int(stream_id), _P(ptr(out) or None),
                                            int(max_frames), _P(ptr(t_frames) or None))


def esi_stream_frame_seq(srv, stream_id: int, seq: int, out):
    """Returns (rc, t_frame_us) for frame number seq of the stream."""
    t = ctypes.c_int64(0)
    rc = _fn("esi_stream_frame_seq")(srv, int(stream_id), int(seq), _P(ptr(out) or None),
                                     ctypes.byref(t))
    return rc, int(t.value)


def esi_bin_events(width: int, height: int, shape: esi_tuning, ring, ring_capacity: int,
                   first: int, n: int, t_base: int, records, runs, cuda_stream=0):
    """Returns (rc, events dropped)."""
    d = ctypes.c_uint64(0)
    rc = _fn("esi_bin_events")(int(width), int(height), ctypes.byref(shape),
                               _P(ptr(ring) or None), int(ring_capacity), int(first), int(n),
                               int(t_base), _P(ptr(records) or None), _P(ptr(runs) or None),
                               ctypes.byref(d), _P(int(cuda_stream) or None))
    return rc, int(d.value)


def esi_stream_state(srv, stream_id: int, S, T) -> int:
    return _fn("esi_stream_state")(srv, int(stream_id), _P(ptr(S) or None), _P(ptr(T) or None))


def esi_stream_close(srv, stream_id: int) -> int:
    return _fn("esi_stream_close")(srv, int(stream_id))


def esi_server_trace(srv):
    """(rc, numpy structured array of the kept tick records, oldest first)."""
    import numpy as np
    n = _sz(0)
    rc = _fn("esi_server_trace")(srv, None, 0, ctypes.byref(n))
    if rc != ESI_OK:
        return rc, None
    buf = (esi_tick_trace * max(n.value, 1))()
    rc = _fn("esi_server_trace")(srv, ctypes.cast(buf, _P), n.value, ctypes.byref(n))
    if rc != ESI_OK:
        return rc, None
    dt = np.dtype([("call_ns", np.int64), ("issued_ns", np.int64), ("ready_ns", np.int64),
                   ("copy_ms", np.float32), ("kernels_ms", np.float32), ("gap_ms", np.float32),
                   ("frames", np.int32), ("events", np.int64), ("streams", np.int32),
                   ("items", np.int32)], align=True)
    assert dt.itemsize == ctypes.sizeof(esi_tick_trace)
    return ESI_OK, np.frombuffer(bytes(buf)[:n.value * dt.itemsize], dtype=dt).copy()


def esi_server_last_error(srv) -> str:
    return (_fn("esi_server_last_error")(srv) or b"").decode()


def esi_server_sync(srv) -> int:
    return _fn("esi_server_sync")(srv)


def esi_server_get_stats(srv):
    st = esi_server_stats()
    rc = _fn("esi_server_get_stats")(srv, ctypes.byref(st))
    return rc, st


def esi_server_reset_stats(srv) -> int:
    return _fn("esi_server_reset_stats")(srv)


def esi_server_destroy(srv) -> None:
    _fn("esi_server_destroy")(srv)


class EsiError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {esi_strerror(code)} ({code})")
        self.code = code


def check(rc: int, what: str = "esi call") -> None:
    if rc != ESI_OK:
        raise EsiError(rc, what)


def make_params(C: float, k_per_s: float, b: float, s_min: float, s_max: float,
                t_origin_us: int = 0, render_decay: int = 0,
                method: int = 0) -> esi_params:
    p = esi_params()
    p.C, p.k_per_s, p.b, p.s_min, p.s_max = C, k_per_s, b, s_min, s_max
    p.t_origin_us, p.render_decay, p.method = int(t_origin_us), int(render_decay), int(method)
    return p
