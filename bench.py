#!/usr/bin/env python3
"""Throughput of the ESI hot path on one GB300 (events/s and frames/s).

Workload (one step): the 640x480, 2 s synthetic stream of configuration 1
(40 Gaussian blobs, per-pixel C ~ N(0.15, 0.03), ~10 M events, int64 us),
rendered as 200 frames of 10 ms with the decay view (render_decay = 1),
C = 0.15, k = 10 /s, b = 2, clamp [-1, 1].  Step k replays the stream shifted
by k * 2 s, so the state carries on as one continuous stream.

value: events/s with every step's events already resident in device memory
(pushed before the timed region), frames written to device memory; inputs
per step (160 MB) exceed the 129 MB L2.  e2e: the same metric through the C
ABI with pinned host buffers inside the timed region: each step pushes its
events from host memory and renders its frames into a host buffer, the next
step's push overlapping this step's render (the synchronous variant is
reported beside it).  With --gpus N (torchrun) every rank runs its own replica
on its own GPU (no collective on the data path; weak scaling).

Further legs on rank 0 (skipped with --no-extras): single-frame latency;
serving of 64 streams of 346x260 and of 192 mixed-resolution streams with
joins and leaves, batched and plain; the 346x260 sinusoid and the 1280x720
checkerboard workloads with the default and the autotuned launch shape; the
Fig. 4 diagnostics and per-event states; the oracle on one host core and on
all of them.

--impl reference times the FP64 CPU oracle (the test reference) on the host
cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "events/s and frames/s at 1 GB300 (% HBM roofline); p50/p99 frame latency, batched vs plain"
WINDOW_US = 10_000
DURATION_US = 2_000_000
PARAMS = dict(C=0.15, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, t_origin_us=0,
              render_decay=1)
WORKLOAD = "blobs 640x480, 2 s, ~10M events (40 Gaussian blobs), 200 x 10 ms frames, decay view"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the same launch shape (4 M events, 80 frames per launch);
# profiles/esi_tile_kernel_blobs640x480_small.md, profiles/esi_bin_kernel_blobs640x480_small.md.
NCU_TRAFFIC_PER_LAUNCH = {"esi_tile": 38525696, "esi_bin": 67803648}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["esi", "reference"], default="esi")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e, latency and CPU-baseline legs")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the two serving legs and print their JSON")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run the small profiling case (0.4 s of the stream, 40 frames, 3 renders) "
                         "and print no bench line; for ncu captures")
    ap.add_argument("--diagnostics-only", action="store_true",
                    help="run only the diagnostics leg (event counts, per-event states, noise "
                         "map) and print its JSON; also the case for their ncu captures")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The step time of the slowest rank (every rank gets it)."""
    if ws == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, steps: int, ws: int, ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return units_per_rank_step * steps * ws / (ms / 1e3)


def make_stream():
    import synth
    sc = synth.blobs_640x480()
    return sc, synth.generate(sc)


def shifted(ev, k):
    e = ev.copy()
    e["t"] += k * DURATION_US
    return e


def frame_times(k, n_windows):
    return np.arange(1, n_windows + 1, dtype=np.int64) * WINDOW_US + k * DURATION_US


def cpu_baseline(sc, ev, budget_s: float = 10.0):
    """The oracle as it stands on one host core: whole-stream replays until budget_s."""
    import oracle
    reps, used, t0 = 0, 0, time.perf_counter()
    n_windows = DURATION_US // WINDOW_US
    while True:
        st = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**PARAMS))
        _, u = st.replay(ev, frame_times(0, n_windows))
        used += u
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 8:
            break
    dt = time.perf_counter() - t0
    return {"value": used / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} replay(s) of the whole 2 s stream ({len(ev)} events, "
                      f"{n_windows} frames each), {dt:.1f} s"}


def _oracle_band(job):
    """Worker: the oracle over the events of one band of rows (pixels of
    different bands never interact, Eq. 5), timed inside the worker."""
    band, n_bands, path, W, H = job
    import oracle
    ev = np.load(path, mmap_mode="r")
    y0, y1 = band * H // n_bands, (band + 1) * H // n_bands
    sel = np.array(ev[(ev["y"] >= y0) & (ev["y"] < y1)])
    sel["y"] -= y0     # the band as a sensor of its own: only its pixels render
    st = oracle.OracleState(W, y1 - y0, oracle.OracleParams(**PARAMS))
    t0 = time.perf_counter()
    _, used = st.replay(sel, frame_times(0, DURATION_US // WINDOW_US))
    return used, time.perf_counter() - t0


def cpu_baseline_parallel(sc, ev):
    """The same oracle on every host core: one process per band of rows
    (spawned, so no CUDA state is inherited); throughput = all events / the
    slowest band's compute time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    try:
        np.save(path, ev)
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_band, [(b, cores, path, sc.W, sc.H) for b in range(cores)])
    finally:
        os.unlink(path)
    used = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return {"value": used / slowest, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole 2 s stream ({used} events, 200 frames) split into {cores} "
                      f"bands of rows, one process each; {slowest:.2f} s for the slowest band"}


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    sc, ev = make_stream()
    # each step: the first 0.4 s of the stream (40 frames) from a fresh state
    n_w = 40
    sample = ev[ev["t"] <= n_w * WINDOW_US]
    tf = frame_times(0, n_w)

    def step():
        st = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**PARAMS))
        st.replay(sample, tf)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = len(sample) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "first 0.4 s (40 frames) per step"},
        "frames_per_s": n_w * args.steps / dt,
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
                         "sample": f"first 0.4 s of the stream ({len(sample)} events, "
                                   f"{n_w} frames) per step"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_esi(args):
    import torch
    import torch.distributed as dist

    from paper_2508_02238_gb300 import esi

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    esi.load_library(build_if_missing=True)

    sc, ev = make_stream()
    n_ev = len(ev)
    n_windows = DURATION_US // WINDOW_US
    P = sc.W * sc.H
    stream = torch.cuda.Stream()
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**PARAMS), stream.cuda_stream)
    esi.check(rc, "esi_create")
    out = torch.empty((n_windows, sc.H, sc.W), dtype=torch.uint8, device="cuda")

    # device-resident inputs: every step's events pushed before timing
    total_steps = args.warmup + args.steps
    for k in range(total_steps):
        esi.check(esi.esi_push_events(h, shifted(ev, k), n_ev, 0), "push")
    tfs = [frame_times(k, n_windows) for k in range(total_steps)]

    def step(k):
        esi.check(esi.esi_render_frames(h, tfs[k], n_windows, out, 1), "render")

    for k in range(args.warmup):
        step(k)
    esi.check(esi.esi_synchronize(h), "sync")
    rc, st0 = esi.esi_get_stats(h)
    esi.check(esi.esi_profile_reset(h))
    esi.check(esi.esi_profile_enable(h, 1))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup, total_steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    esi.check(esi.esi_profile_enable(h, 0))
    rc, prof = esi.esi_profile_read(h)
    rc, st1 = esi.esi_get_stats(h)
    launches = int(st1.kernel_launches - st0.kernel_launches)

    value = whole_job_rate(n_ev, args.steps, ws, ms)
    frames_per_s = whole_job_rate(n_windows, args.steps, ws, ms)

    # roofline of the dominant kernel (algorithmic bytes / measured duration)
    peak, peak_kind = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = None
    step_bytes = 16 * n_ev + 24 * P + n_windows * P
    if dom:
        name, (nl, tot_ms) = dom
        if name == "esi_bin":
            bytes_per_launch = 16.0 * n_ev * args.steps / nl
        else:
            bytes_per_launch = (24.0 * P * nl + n_windows * P * args.steps) / nl
        achieved = bytes_per_launch / (tot_ms / nl / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "peak_kind": f"of {peak_kind}", "unit": "GB/s", "frac": achieved / peak,
                "traffic": NCU_TRAFFIC_PER_LAUNCH.get(name), "launches": nl,
                "avg_launch_us": tot_ms / nl * 1e3, "bytes_per_launch": bytes_per_launch}
    kernels = {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / max(1e-9, sum(x[1] for x in prof.values()))}
               for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator, 640x480 blob scene), state FP32, times int64 us",
        "config": {"workload": WORKLOAD, "events_per_step": n_ev, "frames_per_step": n_windows,
                   "sensor": f"{sc.W}x{sc.H}", "params": PARAMS,
                   "l2": "inputs larger than L2 (160 MB of events per step)",
                   "parallelism": f"replicas x{ws}"},
        "frames_per_s": frames_per_s,
        "roofline": roof,
        "step_roofline": {"bytes_per_step": step_bytes,
                          "achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9,
                          "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
                          "note": "16 B/event + S,T read and written once + 1 B/pixel/frame"},
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clk,
    }

    if not args.no_extras and rank == 0:
        line["e2e"] = e2e_leg(esi, torch, h, stream, sc, ev, out, total_steps, args.steps, n_windows)
        line["latency"] = latency_leg(esi, torch, sc, ev)
        line["serving"] = serving_leg(esi)
        line["serving_mixed"] = mixed_serving_leg(esi)
        line["other_workloads"] = other_workloads_leg(esi, torch)
        line["diagnostics"] = diagnostics_leg(esi, torch)
    elif not args.no_extras:
        line["e2e"] = None
    esi.esi_destroy(h)
    if rank == 0 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(sc, ev)
        line["cpu_baseline_all_cores"] = cpu_baseline_parallel(sc, ev)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e_leg(esi, torch, h, stream, sc, ev, out, k0, steps, n_windows):
    """Steps through the public API with pinned host input and output.

    Pipelined (the reported value): each step pushes its events from host
    memory (the call returns once they are on the device) and queues its
    render into a host buffer (out_on_device = 2), so the next step's push
    overlaps this step's render; one esi_synchronize ends the timed region.
    Synchronous (reported beside it): each render waits for its frames."""
    n_ev = len(ev)
    steps = min(steps, 6)   # distinct pinned inputs: 2 x steps + 4 of 160 MB each
    host_in = []
    for i in range(2 * steps + 4):
        buf = torch.empty(n_ev * 16, dtype=torch.uint8, pin_memory=True)
        buf.numpy().view(ev.dtype)[:] = shifted(ev, k0 + i)
        host_in.append(buf)
    host_out = [torch.empty((n_windows, sc.H, sc.W), dtype=torch.uint8, pin_memory=True)
                for _ in range(2)]

    def step(i, mode):
        esi.check(esi.esi_push_events(h, host_in[i], n_ev, 0), "push")
        esi.check(esi.esi_render_frames(h, frame_times(k0 + i, n_windows), n_windows,
                                        host_out[i % 2], mode), "render")

    def run(first, mode):
        t0 = time.perf_counter()
        for i in range(first, first + steps):
            step(i, mode)
        esi.check(esi.esi_synchronize(h), "sync")
        return time.perf_counter() - t0

    step(0, 0)  # warm, both modes
    step(1, 2)
    step(2, 2)
    esi.check(esi.esi_synchronize(h), "sync")
    torch.cuda.synchronize()
    dt = run(3, 2)
    dt_sync = run(3 + steps, 0)
    return {"value": n_ev * steps / dt, "unit": "events/s",
            "h2d_bytes_per_step": n_ev * 16, "d2h_bytes_per_step": n_windows * sc.W * sc.H,
            "frames_per_s": n_windows * steps / dt,
            "mode": "pipelined: push of step k+1 overlaps the render of step k (out_on_device=2)",
            "synchronous": {"value": n_ev * steps / dt_sync, "unit": "events/s",
                            "mode": "each render waits for its frames (out_on_device=0)"}}


def latency_leg(esi, torch, sc, ev):
    """Plain single-stream path: one 10 ms packet pushed, one frame rendered to host."""
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**PARAMS), 0)
    esi.check(rc)
    out = np.empty((sc.H, sc.W), dtype=np.uint8)
    n_windows = DURATION_US // WINDOW_US
    cuts = np.searchsorted(ev["t"], np.arange(0, n_windows + 1) * WINDOW_US, side="right")
    lat = []
    for w in range(n_windows):
        pkt = np.ascontiguousarray(ev[cuts[w]:cuts[w + 1]])
        t0 = time.perf_counter()
        esi.check(esi.esi_push_events(h, pkt, len(pkt), 0))
        esi.check(esi.esi_render_frame(h, (w + 1) * WINDOW_US, out, 0))
        lat.append((time.perf_counter() - t0) * 1e3)
    esi.esi_destroy(h)
    lat = np.array(lat[5:])
    return {"path": "plain: push 10 ms packet (host) + render one frame (host out)",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "frames": int(len(lat))}


SERVING_STREAMS = 64
SERVING_SECONDS = 0.25


def serving_workload(n_streams=SERVING_STREAMS, seconds=SERVING_SECONDS, seed=1003):
    """64 sinusoid form 346x260 streams, lognormal rates, Poisson packets (1 ms mean)."""
    import synth
    rates = synth.lognormal_rates(n_streams, seed)
    streams = []
    rng = np.random.default_rng(seed)
    for i in range(n_streams):
        sc = synth.serving_stream(i, float(rates[i]), seconds)
        ev = synth.generate(sc)
        # Poisson packet arrivals (mean 1 ms); a packet carries the events since the last one
        gaps = rng.exponential(1000.0, size=int(seconds * 1e6 / 1000) * 3 + 10)
        arr = np.cumsum(gaps).astype(np.int64) + 1
        arr = arr[arr < int(seconds * 1e6)]
        arr = np.append(arr, int(seconds * 1e6))
        cuts = np.searchsorted(ev["t"], arr, side="right")
        streams.append((sc.W, sc.H, ev, arr, cuts))
    return rates, streams


def build_packets(esi, streams, ids):
    import ctypes
    items = []
    for k, (W, H, ev, arr, cuts) in enumerate(streams):
        lo = 0
        base = ev.ctypes.data
        for a, hi in zip(arr, cuts):
            items.append((int(a), ids[k], base + lo * 16, int(hi - lo)))
            lo = int(hi)
    items.sort(key=lambda x: (x[0], x[1]))
    pk = (esi.esi_packet * len(items))()
    for j, (a, sid, ptr_, n) in enumerate(items):
        pk[j].stream, pk[j].arrival_us, pk[j].ev, pk[j].n = sid, a, ptr_, n
    return pk, len(items)


def serving_leg(esi):
    """Batched (one graph per tick) vs plain (per-stream launches), wall-clock paced."""
    rates, streams = serving_workload()
    t_end = int(SERVING_SECONDS * 1e6)
    n_ev = int(sum(len(s[2]) for s in streams))
    params = esi.make_params(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
    out = {"workload": f"{len(streams)} streams 346x260 (sinusoid form), lognormal rates "
                       f"{rates.min() / 1e6:.2f}-{rates.max() / 1e6:.2f} Mev/s (median "
                       f"{np.median(rates) / 1e6:.2f}), Poisson packets 1 ms, 100 frames/s, "
                       f"{SERVING_SECONDS} s", "events": n_ev}
    for mode in ("batched", "batched_throughput"):
        rc, srv = esi.esi_server_create(1 << 30, None, 0)
        esi.check(rc, "server")
        ids = []
        for W, H, *_ in streams:
            rc, sid = esi.esi_stream_open(srv, W, H, params)
            esi.check(rc, "open")
            ids.append(sid)
        pk, npk = build_packets(esi, streams, ids)
        realtime = 1 if mode == "batched" else 0
        t0 = time.perf_counter()
        esi.check(esi.esi_server_run(srv, pk, npk, 1000, t_end, realtime), "run")
        dt = time.perf_counter() - t0
        rc, st = esi.esi_server_get_stats(srv)
        esi.esi_server_destroy(srv)
        out[mode] = {"frames": int(st.frames), "expected_frames": len(streams) * (t_end // 10000),
                     "frame_latency_p50_ms": st.frame_latency_p50_ms,
                     "frame_latency_p99_ms": st.frame_latency_p99_ms,
                     "packet_to_frame_p50_ms": st.packet_latency_p50_ms,
                     "packet_to_frame_p99_ms": st.packet_latency_p99_ms,
                     "gpu_ms_per_tick": st.gpu_ms_per_tick,
                     "kernel_launches_per_tick": int(st.kernel_launches_per_tick),
                     "wall_s": dt, "events_per_s": n_ev / dt if realtime == 0 else None,
                     "frames_per_s": st.frames / dt}
    pk, npk = build_packets(esi, streams, list(range(len(streams))))
    rc, st = esi.esi_plain_run([s[0] for s in streams], [s[1] for s in streams],
                               [params] * len(streams), pk, npk, 1000, t_end, 10000, 1)
    esi.check(rc, "plain")
    out["plain"] = {"frames": int(st.frames), "frame_latency_p50_ms": st.frame_latency_p50_ms,
                    "frame_latency_p99_ms": st.frame_latency_p99_ms,
                    "packet_to_frame_p50_ms": st.packet_latency_p50_ms,
                    "packet_to_frame_p99_ms": st.packet_latency_p99_ms}
    return out


def other_workloads_leg(esi, torch):
    """Device-resident throughput of the other single-stream workloads, measured
    as the main step: K replays of the stream shifted in time, pushed before
    timing, rendered to device memory, CUDA events on the handle's stream."""
    import synth
    peak, _ = load_peaks()
    out = {}
    cases = [("sinusoid 346x260, 1 s, ~1 M events, 100 x 10 ms frames", synth.sinusoid_346x260, 10_000, 12),
             ("checkerboard 1280x720, 1 s, ~50 M events, 100 x 10 ms frames",
              synth.checkerboard_1280x720, 10_000, 3),
             ("checkerboard 1280x720, 1 s, ~50 M events, 1000 x 1 ms frames",
              synth.checkerboard_1280x720, 1_000, 3)]
    streams = {}
    for label, make, win, K in cases:
        if make not in streams:
            sc = make()
            streams[make] = (sc, synth.generate(sc))
        sc, ev = streams[make]
        n_ev = len(ev)
        span = int(round(sc.duration_s * 1e6))
        n_w = span // win
        prm = dict(PARAMS, C=0.2)
        P = sc.W * sc.H
        step_bytes = 16 * n_ev + 24 * P + n_w * P
        fr = torch.empty((n_w, sc.H, sc.W), dtype=torch.uint8, device="cuda")
        tfs = [np.arange(1, n_w + 1, dtype=np.int64) * win + k * span for k in range(1 + K)]
        res = {"events_per_step": n_ev, "frames_per_step": n_w, "steps": K}
        for mode in ("default", "autotuned"):
            st = torch.cuda.Stream()
            rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), st.cuda_stream)
            esi.check(rc, "esi_create")
            if mode == "autotuned":
                # a quarter of the stream as the sample, with its own frame times
                samp = ev[ev["t"] < span // 4]
                stf = np.arange(1, span // 4 // win + 1, dtype=np.int64) * win
                rc, t = esi.esi_autotune(h, samp, len(samp), stf, len(stf), 0)
                esi.check(rc, "autotune")
                res["autotuned_shape"] = {f: getattr(t, f) for f in (
                    "tile_w", "tile_h", "chunk_events", "batch_records", "max_batch_events")}
            for k in range(1 + K):
                e = ev.copy()
                e["t"] += k * span
                esi.check(esi.esi_push_events(h, e, n_ev, 0), "push")
            esi.check(esi.esi_render_frames(h, tfs[0], n_w, fr, 1), "render")
            esi.check(esi.esi_synchronize(h), "sync")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for k in range(1, 1 + K):
                esi.check(esi.esi_render_frames(h, tfs[k], n_w, fr, 1), "render")
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            esi.esi_destroy(h)
            res[mode] = {"ms_per_step": ms, "events_per_s": n_ev / (ms / 1e3),
                         "frames_per_s": n_w / (ms / 1e3),
                         "step_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak}
        out[label] = res
    return out


def diagnostics_leg(esi, torch, reps=5):
    """Fig. 4 diagnostics: per-pixel event counts of the 1280x720 checkerboard's 1 s stream
    (events and counts on the device) and the noise map ln(1 + |S|) of a
    4000x3000 state.  Each launch is timed by the library's CUDA events on
    the handle's stream, with a 256 MB write before it to flush L2."""
    import synth
    peak, _ = load_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}

    def timed(h, st, call, kind):
        esi.check(call(), kind)                      # warm-up
        esi.check(esi.esi_profile_reset(h))
        esi.check(esi.esi_profile_enable(h, 1))
        for _ in range(reps):
            with torch.cuda.stream(st):
                flush.zero_()
            esi.check(call(), kind)
        esi.check(esi.esi_profile_enable(h, 0))
        rc, prof = esi.esi_profile_read(h)
        nl, tot = prof[kind]
        return tot / nl

    sc = synth.checkerboard_1280x720()
    ev = synth.generate(sc)
    n = len(ev)
    st = torch.cuda.Stream()
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**PARAMS), st.cuda_stream)
    esi.check(rc, "esi_create")
    dev_ev = torch.from_numpy(ev.view(np.uint8)).cuda()
    counts = torch.empty(sc.W * sc.H, dtype=torch.int32, device="cuda")
    ms = timed(h, st, lambda: esi.esi_count_events(h, dev_ev, n, 1, counts, 1), "esi_count")
    esi.esi_destroy(h)
    gbs = 16.0 * n / (ms / 1e3) / 1e9
    out["event_counts"] = {"workload": f"checkerboard {sc.W}x{sc.H}, {n} events", "ms": ms,
                           "events_per_s": n / (ms / 1e3), "achieved_gbs": gbs,
                           "frac": gbs / peak, "bytes": "16 B per event read"}
    del dev_ev, counts
    # continuous-time output: S after every event of the main step's stream
    sc1, ev1 = make_stream()
    n1 = len(ev1)
    rc, h = esi.esi_create(sc1.W, sc1.H, esi.make_params(**PARAMS), st.cuda_stream)
    esi.check(rc, "esi_create")
    vals = torch.empty(n1, dtype=torch.float32, device="cuda")
    steps = []
    for k in range(1 + reps):
        esi.check(esi.esi_push_events(h, shifted(ev1, k), n1, 0), "push")
        with torch.cuda.stream(st):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc, m = esi.esi_event_states(h, vals, n1, 1)
        esi.check(rc, "event_states")
        e1.record(st)
        torch.cuda.synchronize()
        if k:
            steps.append(e0.elapsed_time(e1))
    esi.esi_destroy(h)
    ms = float(np.median(steps))
    out["event_states"] = {"workload": f"blobs {sc1.W}x{sc1.H}, {n1} events per call",
                           "ms": ms, "events_per_s": n1 / (ms / 1e3),
                           "note": "binning + the tile kernel with per-event output; S written per event (4 B)"}
    del vals
    W, H = 4000, 3000
    rc, h = esi.esi_create(W, H, esi.make_params(**PARAMS), st.cuda_stream)
    esi.check(rc, "esi_create")
    nmap = torch.empty(W * H, dtype=torch.float32, device="cuda")
    ms = timed(h, st, lambda: esi.esi_noise_map(h, nmap, 1), "esi_noise_map")
    esi.esi_destroy(h)
    gbs = 8.0 * W * H / (ms / 1e3) / 1e9
    out["noise_map"] = {"workload": f"{W}x{H} state", "ms": ms, "achieved_gbs": gbs,
                        "frac": gbs / peak, "bytes": "4 B per pixel read + 4 B written"}
    return out


MIXED_SECONDS = 0.25


def mixed_serving_leg(esi, seconds=MIXED_SECONDS, seed=1004):
    """Mixed resolutions with join/leave: 16 x 1280x720 (checkerboard form), 48 x
    640x480 (blob form), 128 x 346x260 (sinusoid form) streams, lognormal
    rates in [0.1, 20] Mev/s, Poisson packets (1 ms mean), a quarter joining in
    the first half and a fifth leaving in the second, admission by state
    memory, tile height autotuned per sensor size, 100 frames/s per stream."""
    import ctypes
    import synth
    ws = synth.mixed_serving(duration_s=seconds, seed=seed)
    t_end = int(round(seconds * 1e6))
    rng = np.random.default_rng(seed + 1)
    evs = [synth.generate(w["scene"]) for w in ws]
    params = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)
    budget = 768 << 20
    opts = esi.esi_server_opts()
    opts.use_graph, opts.max_streams = 1, 256

    # autotuned tile height per sensor size, on 50 ms of its median-rate stream
    tile_h = {}
    rc, srv = esi.esi_server_create(budget, opts, 0)
    esi.check(rc, "server")
    for dims in sorted({(w["W"], w["H"]) for w in ws}):
        idx = [i for i, w in enumerate(ws) if (w["W"], w["H"]) == dims]
        med = sorted(idx, key=lambda i: ws[i]["rate"])[len(idx) // 2]
        ev = evs[med]
        samp = ev[ev["t"] < ws[med]["t_join_us"] + 50_000]
        rc, sid = esi.esi_stream_open(srv, dims[0], dims[1], esi.make_params(**params))
        esi.check(rc, "open")
        rc, th = esi.esi_stream_autotune(srv, sid, samp, len(samp), 0)
        esi.check(rc, "autotune")
        tile_h[f"{dims[0]}x{dims[1]}"] = th
        esi.check(esi.esi_stream_close(srv, sid), "close")
    esi.esi_server_destroy(srv)

    specs = []
    items = []
    for k, w in enumerate(ws):
        sp = esi.esi_stream_spec()
        sp.width, sp.height = w["W"], w["H"]
        sp.tile_h = tile_h[f"{w['W']}x{w['H']}"]
        sp.params = esi.make_params(**params, t_origin_us=w["t_join_us"])
        specs.append(sp)
        t0, t1 = w["t_join_us"], w["t_leave_us"] if w["t_leave_us"] is not None else t_end
        items.append((t0, 0, k, ctypes.addressof(sp), 0, esi.ESI_PACKET_OPEN))
        gaps = rng.exponential(1000.0, size=int((t1 - t0) / 1000) * 3 + 10)
        arr = t0 + np.cumsum(gaps).astype(np.int64) + 1
        arr = np.append(arr[arr < t1], t1)
        ev = evs[k]
        cuts = np.searchsorted(ev["t"], arr, side="right")
        lo = 0
        for a, hi in zip(arr.tolist(), cuts.tolist()):
            items.append((a, 1, k, ev.ctypes.data + lo * 16, hi - lo, esi.ESI_PACKET_EVENTS))
            lo = hi
        if w["t_leave_us"] is not None:
            items.append((t1, 2, k, 0, 0, esi.ESI_PACKET_CLOSE))
    items.sort(key=lambda x: (x[0], x[1], x[2]))
    pk = (esi.esi_packet * len(items))()
    for j, (a, _, k, p_, n, kind) in enumerate(items):
        pk[j].stream, pk[j].kind, pk[j].arrival_us, pk[j].ev, pk[j].n = k, kind, a, p_, n
    n_ev = int(sum(len(e) for e in evs))
    expected = sum(((w["t_leave_us"] if w["t_leave_us"] is not None else t_end) - w["t_join_us"])
                   // 10_000 for w in ws)
    rates = np.array([w["rate"] for w in ws])
    out = {"workload": "mixed: 16 x 1280x720 + 48 x 640x480 + 128 x 346x260 streams "
                       f"({sum(w['W'] * w['H'] for w in ws) / 1e6:.1f} M pixels), lognormal rates "
                       f"{rates.min() / 1e6:.2f}-{rates.max() / 1e6:.2f} Mev/s (sum "
                       f"{rates.sum() / 1e6:.0f} Mev/s), {sum(w['t_join_us'] > 0 for w in ws)} join "
                       f"late, {sum(w['t_leave_us'] is not None for w in ws)} leave, Poisson packets "
                       f"1 ms, 100 frames/s, {seconds} s",
           "events": n_ev, "expected_frames": int(expected), "state_budget_bytes": budget,
           "autotuned_tile_h": tile_h}
    for mode in ("batched", "batched_throughput"):
        for sp in specs:
            sp.stream_id = -1
        rc, srv = esi.esi_server_create(budget, opts, 0)
        esi.check(rc, "server")
        realtime = 1 if mode == "batched" else 0
        t0 = time.perf_counter()
        esi.check(esi.esi_server_run(srv, pk, len(items), 1000, t_end, realtime), "run")
        dt = time.perf_counter() - t0
        rc, st = esi.esi_server_get_stats(srv)
        esi.esi_server_destroy(srv)
        out[mode] = {"frames": int(st.frames), "events": int(st.events),
                     "streams_admitted": int(st.streams_admitted),
                     "streams_refused": int(st.streams_refused),
                     "frame_latency_p50_ms": st.frame_latency_p50_ms,
                     "frame_latency_p99_ms": st.frame_latency_p99_ms,
                     "packet_to_frame_p50_ms": st.packet_latency_p50_ms,
                     "packet_to_frame_p99_ms": st.packet_latency_p99_ms,
                     "gpu_ms_per_tick": st.gpu_ms_per_tick,
                     "kernel_launches_per_tick": int(st.kernel_launches_per_tick),
                     "wall_s": dt, "events_per_s": n_ev / dt if realtime == 0 else None,
                     "frames_per_s": st.frames / dt}
    return out


def ncu_case():
    """A small case of the same launch shape for kernel captures: 0.8 s of the
    640x480 blob stream (about 4 M events, 64 MB, one sub-batch per render as in
    the bench), 80 frames per render, three renders."""
    import torch  # noqa: F401  (CUDA context as in the bench)
    import synth
    from paper_2508_02238_gb300 import esi
    sc = synth.blobs_640x480(duration_s=0.8)
    ev = synth.generate(sc)
    span = 800_000
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**PARAMS), 0)
    esi.check(rc, "create")
    out = torch.empty((80, sc.H, sc.W), dtype=torch.uint8, device="cuda")
    for k in range(3):
        esi.check(esi.esi_push_events(h, _shift(ev, k * span), len(ev), 0))
    for k in range(3):
        tf = np.arange(1, 81, dtype=np.int64) * WINDOW_US + k * span
        esi.check(esi.esi_render_frames(h, tf, 80, out, 1), "render")
    esi.check(esi.esi_synchronize(h))
    esi.esi_destroy(h)
    print(f"ncu case done: {len(ev)} events x 3 renders")


def _shift(ev, dt):
    e = ev.copy()
    e["t"] += dt
    return e


def main():
    args = parse_args()
    if args.ncu_case:
        ncu_case()
        return
    if args.diagnostics_only:
        import torch
        from paper_2508_02238_gb300 import esi
        esi.load_library(build_if_missing=True)
        print(json.dumps({"diagnostics": diagnostics_leg(esi, torch)}), flush=True)
        return
    if args.serving_only:
        import torch  # noqa: F401  (CUDA context as in the bench)
        from paper_2508_02238_gb300 import esi
        esi.load_library(build_if_missing=True)
        print(json.dumps({"serving": serving_leg(esi), "serving_mixed": mixed_serving_leg(esi)}),
              flush=True)
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_esi(args)


if __name__ == "__main__":
    main()
