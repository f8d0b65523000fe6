#!/usr/bin/env python3
"""Throughput of the ESI hot path on one GB300 (events/s and frames/s).

Headline workload (one step): the 1280x720, 1 s synthetic stream of the
checkerboard scene (32 px squares rotating at 2 rad/s, two bursts of 100 Hz
flicker, 0.05 % hot pixels at 1-20 kHz; ~50 M events, int64 us), rendered as
100 frames of 10 ms with the decay view (render_decay = 1), C = 0.2,
k = 10 /s, b = 2, clamp [-1, 1].  It is the largest single-sensor workload.
Step k replays the stream shifted by k seconds, so the state carries on as
one continuous stream.

value: events/s with every step's events already resident in device memory
(pushed before the timed region), frames written to device memory; inputs
per step (800 MB) exceed the 129 MB L2.  e2e: the same metric through the C
ABI with pinned host buffers inside the timed region: each step pushes its
events (8-byte packed; 16-byte events beside it) from host memory and
renders its frames into a host buffer, the next step's push overlapping this
step's render (the synchronous variant is reported beside it).  With --gpus N (torchrun) every rank runs its own replica
on its own GPU (no collective on the data path; weak scaling).

Further legs on rank 0 (skipped with --no-extras): the other single-sensor
workloads (346x260 sinusoid, 640x480 blobs, the 1280x720 stream in 1 ms
frames); single-frame latency; batched serving of 64 streams of 346x260 and of
192 mixed-resolution streams with joins and leaves, batched and plain; the
Fig. 4 diagnostics and per-event states; and the oracle leg: the FP64 oracle
timed on one host core and on all of them, and its results compared with
the GPU's on every workload (the per-workload maximum errors).  A compact
summary closes the line.

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
PARAMS = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, t_origin_us=0,
              render_decay=1)

# name: (label, generator, duration in us, frame period in us, C)
WORKLOADS = {
    "c0": ("sinusoid 346x260, 1 s, ~1 M events, 100 x 10 ms frames", "sinusoid_346x260",
           1_000_000, 10_000, 0.2),
    "c1": ("blobs 640x480, 2 s, ~10 M events (40 Gaussian blobs), 200 x 10 ms frames",
           "blobs_640x480", 2_000_000, 10_000, 0.15),
    "c2": ("checkerboard 1280x720, 1 s, ~50 M events (rotating, flicker bursts, hot pixels), "
           "100 x 10 ms frames", "checkerboard_1280x720", 1_000_000, 10_000, 0.2),
    "c2_1ms": ("checkerboard 1280x720, 1 s, ~50 M events, 1000 x 1 ms frames",
               "checkerboard_1280x720", 1_000_000, 1_000, 0.2),
}
HEADLINE = "c2"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of a full launch of the headline's shape (--ncu-case: its
# second sub-batch, 4.19 M events and 8 frames), keyed by kernel.
NCU_TRAFFIC_PER_LAUNCH = {"esi_tile": 48732160, "esi_bin": 70952448}
# Warp instructions per launch (smsp__inst_executed.sum) from the same capture.
NCU_INST_PER_LAUNCH = {"esi_tile": 53456009}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["esi", "reference"], default="esi")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every leg but the headline measurement")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the two serving legs and print their JSON")
    ap.add_argument("--serving-apply", type=int, choices=[0, 1, 2], default=0,
                    help="esi_server_opts.apply_mode of the serving legs (0: default)")
    ap.add_argument("--serving-seconds", type=float, default=None,
                    help="stream time of the serving legs (default 5 s)")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run the small profiling case (0.25 s of the headline stream, 25 frames, "
                         "3 renders) and print no bench line; for ncu captures")
    ap.add_argument("--scan-chain", type=int, default=0,
                    help="esi_tuning.scan_chain of the --ncu-case handle (0: default; 33: scan off)")
    ap.add_argument("--diagnostics-only", action="store_true",
                    help="run only the diagnostics leg (event counts, per-event states, noise "
                         "map) and print its JSON; also the case for their ncu captures")
    ap.add_argument("--parity-only", action="store_true",
                    help="run only the oracle comparison of every workload and print its JSON")
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


_STREAMS = {}


def workload(name):
    """(scene, events, span_us, frame period, params) of a named workload."""
    import synth
    label, gen, span, win, C = WORKLOADS[name]
    if gen not in _STREAMS:
        sc = getattr(synth, gen)()
        _STREAMS[gen] = (sc, synth.generate(sc))
    sc, ev = _STREAMS[gen]
    return sc, ev, span, win, dict(PARAMS, C=C)


def shifted(ev, dt):
    e = ev.copy()
    e["t"] += dt
    return e


def frame_times(k, span, win):
    return np.arange(1, span // win + 1, dtype=np.int64) * win + k * span


# The dominant kernel of a render step: the tile kernel (about two thirds of
# the device time in the ncu launch list of the headline, where launches are
# serialised).  The live CUDA-event durations cannot name it: the binning
# runs on a low-priority stream beside the tile kernel, and its event-timed
# duration includes the time it waits for SMs the tile kernel holds.
DOMINANT = "esi_tile"


def tile_roofline(prof, P, frames_per_step, steps, n_ev, peak, peak_kind, traffic=None,
                  name=DOMINANT):
    """Roofline of one kernel: algorithmic bytes per launch over its average
    CUDA-event duration.  Tile kernel: 24 B per pixel of state (S, T read and
    written once per launch) + 1 B per pixel per frame; binning: 16 B per
    event read."""
    if not prof or name not in prof:
        return None
    nl, tot_ms = prof[name]
    if name == "esi_bin":
        bytes_per_launch = 16.0 * n_ev * steps / nl
    else:
        bytes_per_launch = (24.0 * P * nl + frames_per_step * P * steps) / nl
    achieved = bytes_per_launch / (tot_ms / nl / 1e3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
            "peak_kind": f"of {peak_kind}", "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "launches": nl, "avg_launch_us": tot_ms / nl * 1e3,
            "bytes_per_launch": bytes_per_launch}


def issue_roofline(roof, clocks, name=DOMINANT):
    """The dominant kernel against the SMs' instruction issue rate (4 warp
    instructions per cycle per SM at the SM clock sampled during the timed
    region): its warp instructions per launch (ncu) over its average launch
    time.  The tile kernel is bound here, not by HBM."""
    inst = NCU_INST_PER_LAUNCH.get(name)
    if not roof or not inst:
        return None
    import torch
    try:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        return None
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 4 * mhz * 1e6 / 1e9
    achieved = inst / (roof["avg_launch_us"] * 1e-6) / 1e9
    return {"bound": "issue", "kernel": name, "achieved": achieved, "peak": peak,
            "unit": "G warp-instructions/s", "frac": achieved / peak,
            "inst_per_launch": inst, "sm_mhz": mhz, "sms": sms,
            "peak_kind": "4 warp instructions per cycle per SM at the sampled SM clock"}


def kernel_shares(prof):
    tot = max(1e-9, sum(x[1] for x in prof.values()))
    return {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / tot} for k, v in prof.items()}


def device_steps(esi, torch, name, warmup, steps, ws=1, clocks_gpu=None, tuning=None):
    """K timed steps of a workload with every step's events resident on the
    device before timing; CUDA events on the handle's stream."""
    sc, ev, span, win, prm = workload(name)
    n_ev, P = len(ev), sc.W * sc.H
    M = span // win
    stream = torch.cuda.Stream()
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), stream.cuda_stream)
    esi.check(rc, "esi_create")
    if tuning is not None:
        esi.check(esi.esi_set_tuning(h, tuning), "tuning")
    out = torch.empty((M, sc.H, sc.W), dtype=torch.uint8, device="cuda")
    total = warmup + steps
    for k in range(total):
        esi.check(esi.esi_push_events(h, shifted(ev, k * span), n_ev, 0), "push")
    tfs = [frame_times(k, span, win) for k in range(total)]
    for k in range(warmup):
        esi.check(esi.esi_render_frames(h, tfs[k], M, out, 1), "render")
    esi.check(esi.esi_synchronize(h), "sync")
    rc, st0 = esi.esi_get_stats(h)
    esi.check(esi.esi_profile_reset(h))
    esi.check(esi.esi_profile_enable(h, 1))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(clocks_gpu) if clocks_gpu is not None else None
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(warmup, total):
        esi.check(esi.esi_render_frames(h, tfs[k], M, out, 1), "render")
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    esi.check(esi.esi_profile_enable(h, 0))
    rc, prof = esi.esi_profile_read(h)
    rc, st1 = esi.esi_get_stats(h)
    rc, tun = esi.esi_get_tuning(h)
    return {"handle": h, "stream": stream, "out": out, "ms": ms, "prof": prof, "clocks": clk,
            "launches": int(st1.kernel_launches - st0.kernel_launches), "n_ev": n_ev, "P": P,
            "M": M, "span": span, "win": win, "total": total, "sc": sc, "ev": ev, "prm": prm,
            "shape": {f: getattr(tun, f) for f in ("tile_w", "tile_h", "chunk_events",
                                                    "batch_records", "max_batch_events")}}


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    sc, ev, span, win, prm = workload(HEADLINE)
    # each step: the first 0.1 s of the stream (10 frames) from a fresh state
    n_w = 10
    sample = ev[ev["t"] <= n_w * win]
    tf = frame_times(0, span, win)[:n_w]

    def step():
        st = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**prm))
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
        "config": {"workload": WORKLOADS[HEADLINE][0], "sample": "first 0.1 s (10 frames) per step"},
        "frames_per_s": n_w * args.steps / dt,
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
                         "sample": f"first 0.1 s of the stream ({len(sample)} events, "
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

    r = device_steps(esi, torch, HEADLINE, args.warmup, args.steps, ws, clocks_gpu=dev)
    ms, n_ev, P, M = r["ms"], r["n_ev"], r["P"], r["M"]
    value = whole_job_rate(n_ev, args.steps, ws, ms)
    frames_per_s = whole_job_rate(M, args.steps, ws, ms)
    peak, peak_kind = load_peaks()
    roof = tile_roofline(r["prof"], P, M, args.steps, n_ev, peak, peak_kind)
    if roof:
        roof["traffic"] = NCU_TRAFFIC_PER_LAUNCH.get(roof["kernel"])
    step_bytes = 16 * n_ev + 24 * P + M * P
    sc = r["sc"]
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator, 1280x720 checkerboard scene), state FP32, "
                "times int64 us",
        "config": {"workload": WORKLOADS[HEADLINE][0], "events_per_step": n_ev,
                   "frames_per_step": M, "sensor": f"{sc.W}x{sc.H}", "params": r["prm"],
                   "launch_shape": r["shape"],
                   "l2": f"inputs larger than L2 ({16 * n_ev / 1e6:.0f} MB of events per step)",
                   "parallelism": f"replicas x{ws}"},
        "frames_per_s": frames_per_s,
        "roofline": roof,
        "roofline_issue": issue_roofline(roof, r["clocks"]),
        "roofline_binning": tile_roofline(r["prof"], P, M, args.steps, n_ev, peak, peak_kind,
                                          traffic=NCU_TRAFFIC_PER_LAUNCH.get("esi_bin"),
                                          name="esi_bin"),
        "step_roofline": {"bytes_per_step": step_bytes,
                          "achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9,
                          "frac": step_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
                          "note": "16 B/event + S,T read and written once + 1 B/pixel/frame"},
        "kernels": kernel_shares(r["prof"]),
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    extras = not args.no_extras and rank == 0
    legs = {}

    def leg(key, fn, *a):
        # a leg that fails is reported in its key; the headline line still prints
        t0 = time.perf_counter()
        try:
            line[key] = fn(*a)
        except Exception as ex:
            line[key] = {"error": f"{type(ex).__name__}: {ex}"}
            print(f"bench: leg {key} failed: {ex!r}", file=sys.stderr, flush=True)
        legs[key] = round(time.perf_counter() - t0, 1)

    if extras:
        leg("e2e", e2e_leg, esi, torch, r, args.steps)
    elif not args.no_extras:
        line["e2e"] = None
    esi.esi_destroy(r["handle"])
    del r
    if extras:
        sec = args.serving_seconds or SERVING_SECONDS
        leg("other_workloads", other_workloads_leg, esi, torch)
        leg("latency", latency_leg, esi)
        leg("serving", serving_leg, esi, sec)
        leg("serving_mixed", mixed_serving_leg, esi, min(sec, MIXED_SECONDS))
        leg("diagnostics", diagnostics_leg, esi, torch)
        # the oracle leg: the oracle timed on the host cores, and its results
        # against the GPU's on every workload
        leg("cpu_baseline", cpu_baseline, HEADLINE)
        leg("cpu_baseline_all_cores", cpu_baseline_parallel, HEADLINE)
        leg("parity", parity_leg, esi, torch)
        line["leg_seconds"] = legs
        line["summary"] = summary(line)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e_leg(esi, torch, r, steps):
    """Steps through the public API with pinned host input and output.

    Pipelined (the reported value): each step pushes its events from host
    memory (the call returns once they are on the device) and queues its
    render into a host buffer (out_on_device = 2), so the next step's push
    overlaps this step's render; one esi_synchronize ends the timed region.
    Synchronous (reported beside it): each render waits for its frames.
    Inputs: 8-byte packed events (esi_push_packed, the reported value) and
    16-byte events (esi_push_events, beside it), three pinned buffers of
    each.  A step's 16-byte buffer is refilled (times shifted) between the
    timed runs, outside the timed region, so a 16-byte run is three steps.
    A packed buffer needs no refill (the shift moves only the push's time
    base) and is free again once its push returns, so a packed run is
    max(3, min(steps, 30)) steps over the three buffers in turn.  Each run ends with
    one esi_synchronize, so it includes the drain of its last render.  Each
    variant is timed in five runs after two warm-up runs; the median run is
    reported (the host link of a shared box varies from run to run), all
    five beside it."""
    import synth
    h, ev, span, win, M, sc = r["handle"], r["ev"], r["span"], r["win"], r["M"], r["sc"]
    n_ev = len(ev)
    k0 = r["total"]
    nb = 3
    host_in = [torch.empty(n_ev * 16, dtype=torch.uint8, pin_memory=True) for _ in range(nb)]
    views = [b.numpy().view(ev.dtype) for b in host_in]
    t0 = int(ev["t"][0])
    words = synth.pack_events(ev, t0)
    host_pk = [torch.empty(n_ev * 8, dtype=torch.uint8, pin_memory=True) for _ in range(nb)]
    for b in host_pk:
        b.numpy().view(np.uint64)[:] = words
    del words
    host_out = [torch.empty((M, sc.H, sc.W), dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    k = [k0]
    # steps per run, by input kind (packed runs capped to keep the leg short)
    per_run = {True: max(nb, min(int(steps), 30)), False: nb}

    def fill(packed):
        if packed:
            return
        for i in range(nb):
            views[i][:] = ev
            views[i]["t"] += (k[0] + i) * span

    def run(mode, packed):
        ns = per_run[packed]
        ts = time.perf_counter()
        for i in range(ns):
            if packed:
                esi.check(esi.esi_push_packed(h, host_pk[i % nb], n_ev, t0 + (k[0] + i) * span, 0),
                          "push")
            else:
                esi.check(esi.esi_push_events(h, host_in[i], n_ev, 0), "push")
            esi.check(esi.esi_render_frames(h, frame_times(k[0] + i, span, win), M,
                                            host_out[i % 2], mode), "render")
        esi.check(esi.esi_synchronize(h), "sync")
        dt = time.perf_counter() - ts
        k[0] += ns
        return dt

    def timed(mode, packed):
        dts = []
        for _ in range(5):
            fill(packed)
            dts.append(run(mode, packed))
        return statistics.median(dts), [round(n_ev * per_run[packed] / x) for x in dts]

    for packed in (False, True):
        for _ in range(2):   # warm (the handle sizes its ring for the overlap here)
            fill(packed)
            run(2, packed)
    res = {}
    for packed in (True, False):
        for mode in (2, 0):
            res[packed, mode] = timed(mode, packed)
    rc, st = esi.esi_get_stats(h)
    pipe = "pipelined: push of step k+1 overlaps the render of step k (out_on_device=2); " \
           "median of 5 runs"
    sync = "each render waits for its frames (out_on_device=0); median of 5 runs"

    def variant(packed, mode, text):
        dt, runs = res[packed, mode]
        return {"value": n_ev * per_run[packed] / dt, "unit": "events/s",
                "runs_events_per_s": runs, "steps_per_run": per_run[packed], "mode": text}

    out = variant(True, 2, pipe)
    out.update({"input": "8-byte packed events from pinned host memory (esi_push_packed)",
                "ring": {"capacity_events": int(st.ring_capacity), "grows": int(st.ring_grows),
                         "push_waits": int(st.push_waits)},
                "h2d_bytes_per_step": n_ev * 8, "d2h_bytes_per_step": M * sc.W * sc.H,
                "frames_per_s": M * per_run[True] / res[True, 2][0], "steps": per_run[True],
                "synchronous": variant(True, 0, sync),
                "events16": dict(variant(False, 2, pipe), h2d_bytes_per_step=n_ev * 16,
                                 input="16-byte events from pinned host memory (esi_push_events)",
                                 synchronous=variant(False, 0, sync))})
    return out


def latency_leg(esi):
    """Plain single-stream path on the headline workload: one 10 ms packet
    pushed from host memory, one frame rendered into host memory."""
    sc, ev, span, win, prm = workload(HEADLINE)
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), 0)
    esi.check(rc)
    out = np.empty((sc.H, sc.W), dtype=np.uint8)
    n_w = span // WINDOW_US
    cuts = np.searchsorted(ev["t"], np.arange(0, n_w + 1) * WINDOW_US, side="right")
    lat = []
    for w in range(n_w):
        pkt = np.ascontiguousarray(ev[cuts[w]:cuts[w + 1]])
        t0 = time.perf_counter()
        esi.check(esi.esi_push_events(h, pkt, len(pkt), 0))
        esi.check(esi.esi_render_frame(h, (w + 1) * WINDOW_US, out, 0))
        lat.append((time.perf_counter() - t0) * 1e3)
    esi.esi_destroy(h)
    lat = np.array(lat[5:])
    return {"path": "plain: push a 10 ms packet (host) + render one frame (host out), "
                    "headline workload",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "frames": int(len(lat))}


def other_workloads_leg(esi, torch, K=6):
    """Device-resident throughput of the other single-sensor workloads,
    measured as the headline (K timed steps after two warm-up steps), with
    their tile-kernel roofline.  The 346x260 workload also runs with the
    autotuner's launch shape."""
    peak, peak_kind = load_peaks()
    out = {}
    for name in ("c0", "c1", "c2_1ms"):
        tunings = [("default", None)]
        if name == "c0":
            sc, ev, span, win, prm = workload(name)
            rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), 0)
            esi.check(rc, "esi_create")
            samp = ev[ev["t"] < span // 4]
            stf = np.arange(1, span // 4 // win + 1, dtype=np.int64) * win
            rc, t = esi.esi_autotune(h, samp, len(samp), stf, len(stf), 0)
            esi.check(rc, "autotune")
            esi.esi_destroy(h)
            tunings.append(("autotuned", t))
        res = {"workload": WORKLOADS[name][0]}
        for mode, tun in tunings:
            r = device_steps(esi, torch, name, 2, 12 if name == "c0" else K, tuning=tun)
            esi.esi_destroy(r["handle"])
            steps = 12 if name == "c0" else K
            ms = r["ms"] / steps
            step_bytes = 16 * r["n_ev"] + 24 * r["P"] + r["M"] * r["P"]
            roof = tile_roofline(r["prof"], r["P"], r["M"], steps, r["n_ev"], peak, peak_kind)
            res[mode] = {"ms_per_step": ms, "events_per_s": r["n_ev"] / (ms / 1e3),
                         "frames_per_s": r["M"] / (ms / 1e3),
                         "step_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak,
                         "dominant": {k: roof[k] for k in ("kernel", "frac", "avg_launch_us")}
                         if roof else None,
                         "launch_shape": r["shape"]}
        res["events_per_step"] = r["n_ev"]
        res["frames_per_step"] = r["M"]
        out[name] = res
    return out


SERVING_SECONDS = 5.0
SERVING_APPLY = 0   # esi_server_opts.apply_mode of the serving legs (0: the server's default)
# tile rows of the mixed workload's streams by scene form (2: 1280x720
# checkerboard, 1: 640x480 blobs, 0: 346x260 sinusoid)
MIXED_TILE_H = {2: 16, 1: 8, 0: 8}
MIXED_SECONDS = 5.0
SERVING_PARAMS = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0, render_decay=1)


# esi_packet as numpy sees it (same layout as the C struct)
PACKET_DTYPE = np.dtype([("stream", "<i4"), ("kind", "<i4"), ("arrival_us", "<i8"),
                         ("ev", "<u8"), ("n", "<u8")])
SCENE_SECONDS = 0.5   # serving scenes are generated this long and repeated in time


def _packets(esi, parts):
    """parts: arrays of PACKET_DTYPE plus an 'order' key (0 open, 1 events,
    2 close) for packets of one arrival time; sorted by (arrival, order,
    stream) into one esi_packet array."""
    allp = np.concatenate([p[0] for p in parts])
    order = np.concatenate([p[1] for p in parts])
    idx = np.lexsort((allp["stream"], order, allp["arrival_us"]))
    allp = np.ascontiguousarray(allp[idx])
    import ctypes
    assert PACKET_DTYPE.itemsize == ctypes.sizeof(esi.esi_packet)
    pk = (esi.esi_packet * len(allp))()
    np.frombuffer(pk, dtype=PACKET_DTYPE)[:] = allp
    return pk, len(allp)


def _event_part(esi, k, ev, arr):
    """One stream's event packets: each arrival carries the events since
    the previous one."""
    cuts = np.searchsorted(ev["t"], arr, side="right")
    lo = np.concatenate([[0], cuts[:-1]])
    p = np.zeros(len(arr), dtype=PACKET_DTYPE)
    p["stream"], p["kind"], p["arrival_us"] = k, esi.ESI_PACKET_EVENTS, arr
    p["ev"] = ev.ctypes.data + lo.astype(np.uint64) * 16
    p["n"] = (cuts - lo).astype(np.uint64)
    return p, np.ones(len(arr), dtype=np.int8)


def _one_packet(esi, k, kind, t, ptr=0):
    p = np.zeros(1, dtype=PACKET_DTYPE)
    p["stream"], p["kind"], p["arrival_us"], p["ev"] = k, kind, t, ptr
    return p, np.array([0 if kind == esi.ESI_PACKET_OPEN else 2], dtype=np.int8)


def serving_64(seconds, scene_s=None):
    """The 64-stream workload: (rates, streams with generated events)."""
    import synth
    rates, streams = synth.serving_streams(64, seconds, scene_s=scene_s)
    for s in streams:
        s["events"] = synth.stream_events(s)
    return rates, streams


def _server_run(esi, srv, pk, npk, t_end, realtime, tick_us=1000):
    rc = esi.esi_server_run(srv, pk, npk, tick_us, t_end, realtime)
    if rc:
        raise RuntimeError(f"esi_server_run: {esi.esi_strerror(rc)}: {esi.esi_server_last_error(srv)}")


def _tick_gaps(esi, srv):
    """From the server's tick trace: the longest wait between two tick calls
    with work, how many exceeded 2 ms (the executor fell behind), and where a
    tick with frames spends its time (p50 / p99 in ms: host packing and
    queueing, the table copy, the kernels, call to completion stamp; and the
    share of ticks whose work queued behind the previous tick's)."""
    rc, tr = esi.esi_server_trace(srv)
    if rc or tr is None or len(tr) < 2:
        return {}
    gaps = np.diff(tr["call_ns"]) / 1e6
    out = {"max_tick_gap_ms": round(float(gaps.max()), 3),
           "tick_gaps_over_2ms": int((gaps > 2.0).sum()),
           "traced_ticks": int(len(tr))}
    f = tr[tr["frames"] > 0]
    if len(f):
        def pp(x):
            return [round(float(np.percentile(x, 50)), 3), round(float(np.percentile(x, 99)), 3)]
        out["frame_ticks_ms(p50,p99)"] = {
            "host": pp((f["issued_ns"] - f["call_ns"]) / 1e6),
            "copy": pp(f["copy_ms"]), "kernels": pp(f["kernels_ms"]),
            "call_to_ready": pp((f["ready_ns"] - f["call_ns"]) / 1e6),
            "queued_share": round(float(np.mean((f["gap_ms"] >= 0) & (f["gap_ms"] < 0.005))), 3)}
    return out


def _stats(st, dt, realtime, n_ev, expected=None):
    d = {"frames": int(st.frames),
         "frame_latency_p50_ms": st.frame_latency_p50_ms,
         "frame_latency_p99_ms": st.frame_latency_p99_ms,
         "packet_to_frame_p50_ms": st.packet_latency_p50_ms,
         "packet_to_frame_p99_ms": st.packet_latency_p99_ms,
         "gpu_ms_per_tick": st.gpu_ms_per_tick,
         "gpu_tick_p99_ms": st.gpu_tick_p99_ms,
         "host_tick_p50_ms": st.host_tick_p50_ms, "host_tick_p99_ms": st.host_tick_p99_ms,
         "kernel_launches_per_tick": int(st.kernel_launches_per_tick),
         "host_pool_peak_mb": round(st.host_pool_peak_bytes / 2**20, 1),
         "ring_grows": int(st.ring_grows),
         "wall_s": dt, "events_per_s": n_ev / dt if not realtime else None,
         "frames_per_s": st.frames / dt}
    if expected is not None:
        d["expected_frames"] = int(expected)
    return d


def serving_leg(esi, seconds=SERVING_SECONDS):
    """Batched (one graph per tick) vs plain (per-stream launches), paced by
    the wall clock, and batched as fast as possible: 64 streams of 346x260
    (each stream's scene generated for SCENE_SECONDS and repeated)."""
    rates, streams = serving_64(seconds, SCENE_SECONDS)
    t_end = int(round(seconds * 1e6))
    n_ev = int(sum(len(s["events"]) for s in streams))
    params = esi.make_params(**SERVING_PARAMS)
    out = {"workload": f"{len(streams)} streams 346x260 (sinusoid form), lognormal rates "
                       f"{rates.min() / 1e6:.2f}-{rates.max() / 1e6:.2f} Mev/s (median "
                       f"{np.median(rates) / 1e6:.2f}), Poisson packets 1 ms, 100 frames/s, "
                       f"{seconds} s", "events": n_ev}
    expected = len(streams) * (t_end // WINDOW_US)
    opts = esi.esi_server_opts()
    opts.use_graph, opts.apply_mode = 1, SERVING_APPLY
    for mode in ("batched", "batched_throughput"):
        rc, srv = esi.esi_server_create(1 << 30, opts, 0)
        esi.check(rc, "server")
        parts = []
        for k, s in enumerate(streams):
            rc, sid = esi.esi_stream_open(srv, s["W"], s["H"], params)
            esi.check(rc, "open")
            parts.append(_event_part(esi, sid, s["events"], s["arrivals"]))
        pk, npk = _packets(esi, parts)
        realtime = 1 if mode == "batched" else 0
        t0 = time.perf_counter()
        _server_run(esi, srv, pk, npk, t_end, realtime)
        dt = time.perf_counter() - t0
        rc, st = esi.esi_server_get_stats(srv)
        tick_gaps = _tick_gaps(esi, srv)
        esi.esi_server_destroy(srv)
        out[mode] = _stats(st, dt, realtime, n_ev, expected)
        out[mode].update(tick_gaps)
    pk, npk = _packets(esi, [_event_part(esi, k, s["events"], s["arrivals"])
                             for k, s in enumerate(streams)])
    t0 = time.perf_counter()
    rc, st = esi.esi_plain_run([s["W"] for s in streams], [s["H"] for s in streams],
                               [params] * len(streams), pk, npk, 1000, t_end, WINDOW_US, 1)
    esi.check(rc, "plain")
    out["plain"] = _stats(st, time.perf_counter() - t0, 1, n_ev, expected)
    return out


def mixed_workload(esi, seconds, sinks=False, scene_s=None):
    """Mixed resolutions with join/leave: 16 x 1280x720 (checkerboard form),
    48 x 640x480 (blob form), 128 x 346x260 (sinusoid form) streams, lognormal
    rates in [0.1, 20] Mev/s, Poisson packets (1 ms mean), a quarter joining
    in the first half and a fifth leaving in the second (scenes generated
    for at most scene_s and repeated).  Returns the workload, its packets,
    specs and per-stream events (and frame sinks)."""
    import ctypes
    import synth
    ws = synth.mixed_serving(duration_s=seconds, scene_s=scene_s)
    arrs = synth.mixed_arrivals(ws, duration_s=seconds)
    t_end = int(round(seconds * 1e6))
    evs = [synth.stream_events(w) for w in ws]
    specs, parts, sink = [], [], []
    tile_h = MIXED_TILE_H
    for k, (w, arr) in enumerate(zip(ws, arrs)):
        sp = esi.esi_stream_spec()
        sp.width, sp.height = w["W"], w["H"]
        sp.tile_h = tile_h[w["form"]]
        sp.params = esi.make_params(**SERVING_PARAMS, t_origin_us=w["t_join_us"])
        t1 = w["t_leave_us"] if w["t_leave_us"] is not None else t_end
        if sinks:
            nf = (t1 - w["t_join_us"]) // WINDOW_US
            buf = np.zeros((max(nf, 1), w["H"], w["W"]), dtype=np.uint8)
            tfs = np.zeros(max(nf, 1), dtype=np.int64)
            sp.frame_sink, sp.sink_frames, sp.sink_t_frames = buf.ctypes.data, nf, tfs.ctypes.data
            sink.append((buf, tfs, nf))
        specs.append(sp)
        parts.append(_one_packet(esi, k, esi.ESI_PACKET_OPEN, w["t_join_us"], ctypes.addressof(sp)))
        parts.append(_event_part(esi, k, evs[k], arr))
        if w["t_leave_us"] is not None:
            parts.append(_one_packet(esi, k, esi.ESI_PACKET_CLOSE, t1))
    pk, npk = _packets(esi, parts)
    return ws, pk, npk, specs, evs, sink


def mixed_serving_leg(esi, seconds=SERVING_SECONDS):
    """Mixed-resolution serving: batched, paced by the wall clock, and as
    fast as possible; 100 frames/s per stream, admission by state memory."""
    t_end = int(round(seconds * 1e6))
    ws, pk, npk, specs, evs, _ = mixed_workload(esi, seconds, scene_s=SCENE_SECONDS)
    budget = 768 << 20
    opts = esi.esi_server_opts()
    opts.use_graph, opts.max_streams, opts.apply_mode = 1, 256, SERVING_APPLY
    opts.host_pool_bytes = 1 << 30
    n_ev = int(sum(len(e) for e in evs))
    expected = sum(((w["t_leave_us"] if w["t_leave_us"] is not None else t_end) - w["t_join_us"])
                   // WINDOW_US for w in ws)
    rates = np.array([w["rate"] for w in ws])
    out = {"workload": "mixed: 16 x 1280x720 + 48 x 640x480 + 128 x 346x260 streams "
                       f"({sum(w['W'] * w['H'] for w in ws) / 1e6:.1f} M pixels), lognormal rates "
                       f"{rates.min() / 1e6:.2f}-{rates.max() / 1e6:.2f} Mev/s (sum "
                       f"{rates.sum() / 1e6:.0f} Mev/s), {sum(w['t_join_us'] > 0 for w in ws)} join "
                       f"late, {sum(w['t_leave_us'] is not None for w in ws)} leave, Poisson packets "
                       f"1 ms, 100 frames/s, {seconds} s",
           "events": n_ev, "state_budget_bytes": budget,
           "tile_h": {"1280x720": MIXED_TILE_H[2], "640x480": MIXED_TILE_H[1],
                      "346x260": MIXED_TILE_H[0]}}
    for mode in ("batched", "batched_throughput"):
        for sp in specs:
            sp.stream_id = -1
        rc, srv = esi.esi_server_create(budget, opts, 0)
        esi.check(rc, "server")
        realtime = 1 if mode == "batched" else 0
        t0 = time.perf_counter()
        _server_run(esi, srv, pk, npk, t_end, realtime)
        dt = time.perf_counter() - t0
        rc, st = esi.esi_server_get_stats(srv)
        tick_gaps = _tick_gaps(esi, srv)
        esi.esi_server_destroy(srv)
        out[mode] = _stats(st, dt, realtime, n_ev, expected)
        out[mode].update(tick_gaps)
        out[mode]["streams_admitted"] = int(st.streams_admitted)
        out[mode]["streams_refused"] = int(st.streams_refused)
    return out


def diagnostics_leg(esi, torch, reps=5):
    """Fig. 4 diagnostics: per-pixel event counts of the 1280x720 checkerboard's 1 s stream
    (events and counts on the device) and the noise map ln(1 + |S|) of a
    4000x3000 state.  Each launch is timed by the library's CUDA events on
    the handle's stream, with a 256 MB write before it to flush L2; per-event
    states of the 640x480 blob stream."""
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

    sc, ev, _, _, prm = workload("c2")
    n = len(ev)
    st = torch.cuda.Stream()
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), st.cuda_stream)
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
    # continuous-time output: S after every event of the 640x480 stream
    sc1, ev1, span1, _, prm1 = workload("c1")
    n1 = len(ev1)
    rc, h = esi.esi_create(sc1.W, sc1.H, esi.make_params(**prm1), st.cuda_stream)
    esi.check(rc, "esi_create")
    vals = torch.empty(n1, dtype=torch.float32, device="cuda")
    steps = []
    for k in range(1 + reps):
        esi.check(esi.esi_push_events(h, shifted(ev1, k * span1), n1, 0), "push")
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


# --------------------------------------------------------------- oracle leg
def cpu_baseline(name, budget_s: float = 10.0):
    """The oracle as it stands on one host core: whole-stream replays until budget_s."""
    import oracle
    sc, ev, span, win, prm = workload(name)
    reps, used, t0 = 0, 0, time.perf_counter()
    tf = frame_times(0, span, win)
    while True:
        st = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**prm))
        _, u = st.replay(ev, tf)
        used += u
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 8:
            break
    dt = time.perf_counter() - t0
    return {"value": used / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} replay(s) of the whole {span / 1e6:g} s stream ({len(ev)} events, "
                      f"{len(tf)} frames each), {dt:.1f} s"}


def _oracle_band(job):
    """Worker: the oracle over the events of one band of rows (pixels of
    different bands never interact, Eq. 5), timed inside the worker."""
    band, n_bands, path, W, H, prm, tf = job
    import oracle
    ev = np.load(path, mmap_mode="r")
    y0, y1 = band * H // n_bands, (band + 1) * H // n_bands
    sel = np.array(ev[(ev["y"] >= y0) & (ev["y"] < y1)])
    sel["y"] -= y0     # the band as a sensor of its own: only its pixels render
    st = oracle.OracleState(W, y1 - y0, oracle.OracleParams(**prm))
    t0 = time.perf_counter()
    _, used = st.replay(sel, tf)
    return used, time.perf_counter() - t0


def cpu_baseline_parallel(name):
    """The same oracle on every host core: one process per band of rows
    (spawned, so no CUDA state is inherited); throughput = all events / the
    slowest band's compute time."""
    import multiprocessing as mp
    sc, ev, span, win, prm = workload(name)
    tf = frame_times(0, span, win)
    cores = os.cpu_count() or 1
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    try:
        np.save(path, ev)
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_band, [(b, cores, path, sc.W, sc.H, prm, tf)
                                          for b in range(cores)])
    finally:
        os.unlink(path)
    used = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return {"value": used / slowest, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole {span / 1e6:g} s stream ({used} events, {len(tf)} frames) split "
                      f"into {cores} bands of rows, one process each; {slowest:.2f} s for the "
                      f"slowest band"}


class ParityAcc:
    """Maximum errors of GPU results against the oracle's, for one workload:
    state error |dS| / max(|S_ref|, C) (the tests' bar, 1e-5) and with the
    floor 1e-3 C, the largest |dS| where |S_ref| < C in units in the last
    place of C in FP32, T exactness, frame LSB differences."""

    def __init__(self):
        self.err_c = self.err_mc = self.ulps_c = 0.0
        self.t_exact = True
        self.lsb = self.off = self.frames = self.pixels = 0

    def state(self, S, T, S_ref, T_ref, C):
        d = np.abs(np.asarray(S, np.float64) - S_ref)
        if d.size:
            self.err_c = max(self.err_c, float(np.max(d / np.maximum(np.abs(S_ref), C))))
            self.err_mc = max(self.err_mc, float(np.max(d / np.maximum(np.abs(S_ref), 1e-3 * C))))
            small = np.abs(S_ref) < C
            if small.any():
                ulp = float(np.spacing(np.float32(C)))
                self.ulps_c = max(self.ulps_c, float(np.max(d[small])) / ulp)
        self.t_exact &= bool(np.array_equal(T, T_ref))
        self.pixels += int(d.size)

    def frames_(self, got, ref):
        d = np.abs(got.astype(np.int16) - ref.astype(np.int16))
        if d.size:
            self.lsb = max(self.lsb, int(d.max()))
            self.off += int(np.count_nonzero(d))
        self.frames += int(got.shape[0]) if got.ndim == 3 else 1

    def out(self):
        return {"state_err": self.err_c, "state_err_floor_1e-3C": self.err_mc,
                "abs_err_near_zero_ulps_of_C": round(self.ulps_c, 2),
                "T_exact": self.t_exact, "frame_max_lsb": self.lsb,
                "frame_off_by_one": self.off, "frames": self.frames, "pixels": self.pixels,
                "pass": self.err_c <= 1e-5 and self.t_exact and self.lsb <= 1}


def parity_leg(esi, torch):
    """The GPU's frames and final state against the FP64 oracle's on every
    workload: the single-sensor ones rendered in one call (the headline's
    launch shape), the 64-stream and the mixed serving workloads served by the
    executor as fast as possible with every frame kept (0.25 s of stream
    time), each stream against the oracle run on it alone."""
    import oracle
    out = {}
    for name in ("c0", "c1", "c2", "c2_1ms"):
        sc, ev, span, win, prm = workload(name)
        tf = frame_times(0, span, win)
        rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**prm), 0)
        esi.check(rc, "esi_create")
        esi.check(esi.esi_push_events(h, ev, len(ev), 0), "push")
        fr = torch.empty((len(tf), sc.H, sc.W), dtype=torch.uint8, device="cuda")
        esi.check(esi.esi_render_frames(h, tf, len(tf), fr, 1), "render")
        S = np.empty(sc.W * sc.H, dtype=np.float32)
        T = np.empty(sc.W * sc.H, dtype=np.int64)
        esi.check(esi.esi_get_state(h, S, T, 0), "state")
        esi.esi_destroy(h)
        # 1 ms frames: every 10th frame is compared, the last one included
        # (the oracle renders only those; its state passes through the same
        # events either way)
        every = 10 if len(tf) > 200 else 1
        got = fr[every - 1::every].cpu().numpy()
        del fr
        ref = oracle.OracleState(sc.W, sc.H, oracle.OracleParams(**prm))
        ref_frames, _ = ref.replay(ev, tf[every - 1::every])
        acc = ParityAcc()
        acc.state(S, T, ref.S, ref.T, prm["C"])
        acc.frames_(got, ref_frames)
        out[name] = acc.out()
        del got, ref_frames
    out["c3"] = _parity_serving_64(esi, oracle)
    out["c4"] = _parity_mixed(esi, oracle)
    return out


def _parity_serving_64(esi, oracle, seconds=0.25):
    rates, streams = serving_64(seconds)
    t_end = int(round(seconds * 1e6))
    nf = t_end // WINDOW_US
    params = esi.make_params(**SERVING_PARAMS)
    rc, srv = esi.esi_server_create(1 << 30, None, 0)
    esi.check(rc, "server")
    parts, sinks, ids = [], [], []
    for s in streams:
        rc, sid = esi.esi_stream_open(srv, s["W"], s["H"], params)
        esi.check(rc, "open")
        buf = np.zeros((nf, s["H"], s["W"]), dtype=np.uint8)
        tfs = np.zeros(nf, dtype=np.int64)
        esi.check(esi.esi_stream_set_frame_sink(srv, sid, buf, nf, tfs), "sink")
        sinks.append((buf, tfs))
        ids.append(sid)
        parts.append(_event_part(esi, sid, s["events"], s["arrivals"]))
    pk, npk = _packets(esi, parts)
    _server_run(esi, srv, pk, npk, t_end, 0)
    acc = ParityAcc()
    for s, sid, (buf, tfs) in zip(streams, ids, sinks):
        S = np.empty(s["W"] * s["H"], dtype=np.float32)
        T = np.empty(s["W"] * s["H"], dtype=np.int64)
        esi.check(esi.esi_stream_state(srv, sid, S, T), "state")
        tf = np.arange(1, nf + 1, dtype=np.int64) * WINDOW_US
        ok_t = np.array_equal(tfs, tf)
        ref = oracle.OracleState(s["W"], s["H"], oracle.OracleParams(**SERVING_PARAMS))
        ev = s["events"]
        ref_frames, used = ref.replay(ev, tf)
        ref.integrate(ev[used:])
        acc.state(S, T, ref.S, ref.T, SERVING_PARAMS["C"])
        acc.frames_(buf, ref_frames)
        acc.t_exact &= ok_t
    esi.esi_server_destroy(srv)
    r = acc.out()
    r["streams"] = len(streams)
    return r


def _parity_mixed(esi, oracle, seconds=0.25):
    t_end = int(round(seconds * 1e6))
    ws, pk, npk, specs, evs, sinks = mixed_workload(esi, seconds, sinks=True)
    opts = esi.esi_server_opts()
    opts.use_graph, opts.max_streams = 1, 256
    opts.host_pool_bytes = 1 << 30
    rc, srv = esi.esi_server_create(768 << 20, opts, 0)
    esi.check(rc, "server")
    _server_run(esi, srv, pk, npk, t_end, 0)
    acc = ParityAcc()
    for w, sp, ev, (buf, tfs, nf) in zip(ws, specs, evs, sinks):
        t0 = w["t_join_us"]
        tf = t0 + np.arange(1, nf + 1, dtype=np.int64) * WINDOW_US
        acc.t_exact &= bool(np.array_equal(tfs[:nf], tf))
        prm = dict(SERVING_PARAMS, t_origin_us=t0)
        ref = oracle.OracleState(w["W"], w["H"], oracle.OracleParams(**prm))
        ref_frames, used = ref.replay(ev, tf)
        acc.frames_(buf[:nf], ref_frames)
        if sp.stream_id >= 0:       # still open: its state too
            S = np.empty(w["W"] * w["H"], dtype=np.float32)
            T = np.empty(w["W"] * w["H"], dtype=np.int64)
            esi.check(esi.esi_stream_state(srv, sp.stream_id, S, T), "state")
            ref.integrate(ev[used:])
            acc.state(S, T, ref.S, ref.T, prm["C"])
    esi.esi_server_destroy(srv)
    r = acc.out()
    r["streams"] = len(ws)
    r["left"] = sum(w["t_leave_us"] is not None for w in ws)
    return r


def summary(line):
    """The numbers to read first, compact (the line's last key)."""
    def g(x, nd=3):
        return None if x is None else round(x / 1e9, nd)

    def lat(d):
        return [round(d[k], 3) for k in ("frame_latency_p50_ms", "frame_latency_p99_ms",
                                          "packet_to_frame_p50_ms", "packet_to_frame_p99_ms")]
    s = {"Gev_s": {HEADLINE: g(line["value"])},
         "tile_frac": {HEADLINE: round(line["roofline"]["frac"], 4) if line.get("roofline") else None},
         "step_frac": {HEADLINE: round(line["step_roofline"]["frac"], 4)},
         "e2e_Gev_s": g(line["e2e"]["value"]) if (line.get("e2e") or {}).get("value") else None,
         "e2e_events16_Gev_s": g(((line.get("e2e") or {}).get("events16") or {}).get("value"))}

    def ok(d):
        return isinstance(d, dict) and "error" not in d
    for name, r in (line.get("other_workloads") if ok(line.get("other_workloads")) else {}).items():
        s["Gev_s"][name] = g(r["default"]["events_per_s"])
        s["step_frac"][name] = round(r["default"]["step_hbm_frac"], 4)
        if r["default"].get("dominant"):
            s["tile_frac"][name] = round(r["default"]["dominant"]["frac"], 4)
    sv = {}
    for key, tag in (("serving", "c3"), ("serving_mixed", "c4")):
        d = line.get(key)
        if not d:
            continue
        if not ok(d):
            sv[tag] = d
            continue
        e = {"lat_ms(f50,f99,p50,p99)": {m: lat(d[m]) for m in ("batched", "plain") if m in d},
             "frames": f"{d['batched']['frames']}/{d['batched'].get('expected_frames')}",
             "max_Gev_s": g(d["batched_throughput"]["events_per_s"])}
        sv[tag] = e
    s["serving"] = sv
    s["parity(err,err1e-3C,ulpsC,lsb,off,frames)"] = {
        k: [float(f"{v['state_err']:.2e}"), float(f"{v['state_err_floor_1e-3C']:.2e}"),
            v.get("abs_err_near_zero_ulps_of_C"), v["frame_max_lsb"], v["frame_off_by_one"], v["frames"]]
        for k, v in (line.get("parity") if ok(line.get("parity")) else {}).items()}
    return s


def ncu_case(scan_chain=0):
    """A small case of the headline's launch shape for kernel captures: the
    first 0.25 s of the 1280x720 stream (about 12 M events, 200 MB, three
    4 M-event sub-batches per render as in the bench), 25 frames per render,
    three renders.  scan_chain: esi_tuning.scan_chain (0: default; 33: the
    segmented scan off)."""
    import torch  # noqa: F401  (CUDA context as in the bench)
    import synth
    from paper_2508_02238_gb300 import esi
    sc = synth.checkerboard_1280x720(duration_s=0.25)
    ev = synth.generate(sc)
    span = 250_000
    rc, h = esi.esi_create(sc.W, sc.H, esi.make_params(**PARAMS), 0)
    esi.check(rc, "create")
    if scan_chain:
        t = esi.esi_tuning()
        t.scan_chain = scan_chain
        esi.check(esi.esi_set_tuning(h, t), "tuning")
    out = torch.empty((25, sc.H, sc.W), dtype=torch.uint8, device="cuda")
    for k in range(3):
        esi.check(esi.esi_push_events(h, shifted(ev, k * span), len(ev), 0))
    for k in range(3):
        tf = np.arange(1, 26, dtype=np.int64) * WINDOW_US + k * span
        esi.check(esi.esi_render_frames(h, tf, 25, out, 1), "render")
    esi.check(esi.esi_synchronize(h))
    esi.esi_destroy(h)
    print(f"ncu case done: {len(ev)} events x 3 renders")


def main():
    global SERVING_APPLY
    args = parse_args()
    SERVING_APPLY = args.serving_apply
    if args.ncu_case:
        ncu_case(args.scan_chain)
        return
    if args.diagnostics_only or args.serving_only or args.parity_only:
        import torch
        from paper_2508_02238_gb300 import esi
        esi.load_library(build_if_missing=True)
        torch.cuda.set_device(0)
        if args.diagnostics_only:
            print(json.dumps({"diagnostics": diagnostics_leg(esi, torch)}), flush=True)
        elif args.serving_only:
            sec = args.serving_seconds or SERVING_SECONDS
            out = {}
            for key, fn in (("serving", serving_leg), ("serving_mixed", mixed_serving_leg)):
                try:
                    out[key] = fn(esi, sec)
                except Exception as ex:
                    out[key] = {"error": f"{type(ex).__name__}: {ex}"}
            print(json.dumps(out), flush=True)
            if any("error" in v for v in out.values()):
                sys.exit(1)
        else:
            print(json.dumps({"parity": parity_leg(esi, torch)}), flush=True)
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_esi(args)


if __name__ == "__main__":
    main()
