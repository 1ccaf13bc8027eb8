#!/usr/bin/env python3
"""Benchmark of the X-engine hot path on B300: full-band Pathfinder integration.

Workload (one "step"): the full 400 MHz CHIME Pathfinder band, N = 256 inputs x F = 1024 channels,
a stream of 64 frames of T = 4096 samples (0.671 s of sky at 390,625 samples/s per channel). Each
frame arrives as 131,072 UDP packets (16-byte header + 8 KiB payload, 128 streams of 8 channels)
already resident in HBM; per frame one xe_correlate_packets call (the frame's index from the
packet headers, then the correlation reading every sample from its packet, lost packets as zeros,
accumulating); at the end of the integration xe_normalize. Inputs are synthetic (seeded noise + 3
point sources, 4+4-bit), 64 distinct frames, ~69 GB of packets: larger than L2.

Prints one JSON line (rank 0). Metric: CMAC/s (complex multiply-accumulates of the upper-triangle
visibilities, F * N(N+1)/2 * T per frame) and the real-time factor.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xe|reference] [--frames 64]
    python bench.py --config 1|2|4|6 [--impl xe|reference]   # the other workloads, frames in HBM

--config 1: N=16, F=4, T=4096 uniform nibbles; 2: the per-server Pathfinder frame N=256, F=64,
T=16384 (signal model); 4: 24 uneven jobs (N 64..2048, F 16..256, T 1024..32768) in one batched
launch; 6: the full-CHIME scale per server, N=2048, F=64, T=16384. For these the step is
correlation + normalisation of frames already in HBM.
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
sys.path.insert(0, ROOT)

N_INPUTS = 256
N_CHAN = 1024
N_TIME = 4096
N_FRAMES = 64
GROUPS_PER_STREAM = 1          # 128 streams of 8 channels (one 10GbE link each)
SAMPLE_RATE = 390625.0         # samples/s per channel: 400 MHz / 1024 channels
METRIC = "X-engine CMAC/s & real-time factor at N=256x1024 ch; int8 pipe %; p99 latency"


def npairs(n):
    return n * (n + 1) // 2


def cmac_per_frame(N=N_INPUTS, F=N_CHAN, T=N_TIME):
    return F * npairs(N) * T


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle (CPU) arm

def cpu_oracle_sample(min_seconds: float = 10.0, max_frames: int = N_FRAMES, channels: int = 16, seed: int = 3):
    """The oracle as it stands on a bounded sample of the workload: `channels` channels (2 streams of
    8) of consecutive frames through oracle assembly, correlation, counts and normalisation, adding
    frames until about `min_seconds` of CPU work. Input generation is not timed."""
    import numpy as np

    import oracle
    import synth

    N, T = N_INPUTS, N_TIME
    lost = np.zeros(channels, np.uint32)
    vis = None
    dt = 0.0
    frames = 0
    for k in range(max_frames):
        if dt >= min_seconds:
            break
        frames += 1
        fr = synth.signal_frame(N, channels, T, seed + k)
        pk = synth.packetize(fr, k * T // 4, GROUPS_PER_STREAM)
        ts = time.perf_counter()
        frame, _, lost, _ = oracle.assemble(pk, k * T // 4, GROUPS_PER_STREAM, N, channels, T, lost=lost)
        v, _ = oracle.correlate(frame)
        vis = v if vis is None else vis + v
        dt += time.perf_counter() - ts
    ts = time.perf_counter()
    n = oracle.counts_from_counters(frames * T, lost, N)
    oracle.normalize(vis, n)
    dt += time.perf_counter() - ts
    cmac = channels * npairs(N) * T * frames
    return {"value": cmac / dt, "unit": "CMAC/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{channels} channels x {frames} frame(s) of T={T}, N={N}: packets -> assemble -> "
                      f"correlate -> counts -> normalise ({dt:.1f} s of CPU work)",
            "seconds": dt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    base = None
    for _ in range(args.steps):
        base = cpu_oracle_sample()
        vals.append(base["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "CMAC/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["seconds"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": workload_config(args),
            "realtime_factor": v / (N_CHAN * npairs(N_INPUTS) * SAMPLE_RATE),
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": v, "unit": "CMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def make_serving_packets(torch, dev, frames_per_stream: int = 8, seed: int = 5000):
    """Configuration 5's packets: 8 F-engine streams x 128 channels (16 groups of 8), N = 256, T = 4096
    per frame, 16-byte-header packets with 8 KiB payloads, 0.1% dropped, 0.5% reordered (displacement
    1..64). Returns, per stream, the packets in arrival order in pinned host memory and in device
    memory, and their headers in host memory."""
    import numpy as np

    import synth

    S, GPS, N, T = 8, 16, 256, 4096
    host, devp, hdrs = [], [], []
    for s in range(S):
        fr = synth.signal_frame_torch(N, 8 * GPS, T * frames_per_stream, seed + s, device=dev, chunk=32)
        pk = synth.packetize_torch(fr, 0, GPS)
        del fr
        pk[:, 0:2] = torch.tensor(list(np.uint16(s).tobytes()), dtype=torch.uint8, device=dev)
        order = synth.network_order(pk.shape[0], seed + 100 + s, p_drop=0.001, p_reorder=0.005)
        pk = pk[torch.from_numpy(order).to(dev)].contiguous()
        h = torch.empty(pk.shape, dtype=torch.uint8).pin_memory()
        h.copy_(pk)
        host.append(h)
        devp.append(pk)
        hdrs.append(np.ascontiguousarray(h[:, :16].numpy()))
    torch.cuda.synchronize(dev)
    return host, devp, hdrs


def link_gbs(torch, dev, nbytes: int = 1 << 30) -> float:
    """Pinned host -> device copy rate (GB/s) of this machine's host link, best of 3."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        d.copy_(h, non_blocking=True)
        e1.record()
        torch.cuda.synchronize(dev)
        best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del h, d
    return best


def run_serving(xe, torch, dev, pk, offered_gbps, feed: str = "host", seed: int = 5000, ring_frames: int = 6,
                frames_per_stream: int = 8):
    """Configuration 5 through xe_stream_*: the 8 streams' packets arrive as Poisson processes
    totalling `offered_gbps` of payload (None: as fast as the producer loop submits them), from
    pinned host memory (feed "host": H2D copies) or from device memory (feed "device": D2D copies,
    headers read from a host copy). Reports the achieved payload rate and the p50 / p99 latency of a
    frame from its close, and from the submission of its last packet, to its normalised visibilities
    being complete."""
    import numpy as np

    import synth

    host, devp, hdrs = pk
    S, GPS, N, T = 8, 16, 256, 4096
    stride = synth.packet_stride(N)
    rng = np.random.default_rng(seed)
    if offered_gbps:
        rate = offered_gbps * 1e9 / 8 / synth.payload_bytes(N) / S         # packets/s per stream
        arrive = [np.cumsum(rng.exponential(1.0 / rate, h.shape[0])) for h in host]
    else:
        arrive = [np.zeros(h.shape[0]) for h in host]
    cfg = xe.StreamCfg(S, GPS, N, T, stride, 1024, ring_frames, 16, 8, 2, 0, 500)
    handle = xe.xe_stream_create(cfg)
    pos = [0] * S
    done = 0
    total = S * frames_per_stream
    flushed = False
    t0 = time.perf_counter()
    try:
        while done < total:
            now = time.perf_counter() - t0
            for s in range(S):
                n_pk = host[s].shape[0]
                if pos[s] >= n_pk:
                    continue
                hi = int(np.searchsorted(arrive[s], now, side="right"))
                while pos[s] < hi:
                    n = min(4096, hi - pos[s])
                    if feed == "host":
                        st = xe.xe_stream_submit(handle, s, host[s].data_ptr() + pos[s] * stride, n)
                    else:
                        st = xe.xe_stream_submit_device(handle, s, devp[s].data_ptr() + pos[s] * stride,
                                                        hdrs[s][pos[s]:pos[s] + n], n)
                    if st != xe.XE_OK:
                        break
                    pos[s] += n
            if not flushed and all(p >= h.shape[0] for p, h in zip(pos, host)):
                flushed = xe.xe_stream_flush(handle) == xe.XE_OK
            r = xe.xe_stream_poll(handle, 0)
            while r is not None:
                xe.xe_stream_release(handle, r)
                done += 1
                r = xe.xe_stream_poll(handle, 0)
            if time.perf_counter() - t0 > 120:
                break
        wall = time.perf_counter() - t0
        st = xe.xe_stream_stats(handle)
    finally:
        xe.xe_stream_destroy(handle)
    payload = sum(int(p) for p in pos) * synth.payload_bytes(N)
    return {"feed": feed, "offered_gbps": offered_gbps, "frames": int(st.frames_done),
            "achieved_gbps": payload * 8 / wall / 1e9, "wall_s": wall,
            "latency_p50_ms": st.latency_p50_us / 1e3, "latency_p99_ms": st.latency_p99_us / 1e3,
            "latency_max_ms": st.latency_max_us / 1e3,
            "latency_from_last_packet_p50_ms": st.latency_submit_p50_us / 1e3,
            "latency_from_last_packet_p99_ms": st.latency_submit_p99_us / 1e3,
            "rounds": int(st.batches), "max_frames_per_round": int(st.max_batch_seen),
            "device_bytes": int(st.device_bytes)}


def run_serving_suite(xe, torch, dev):
    """Configuration 5 at offered loads of 25 / 50 / 80 % of the measured host link, at the paper's
    819.2 Gb/s from host memory (above the link), and from device memory at 819.2 Gb/s and unpaced
    (the loop's own ceiling)."""
    link = link_gbs(torch, dev)
    pk = make_serving_packets(torch, dev)
    link_payload_gbps = link * 8 * 8192 / 8208                     # payload share of the records
    rows = []
    for frac in (0.25, 0.5, 0.8):
        r = run_serving(xe, torch, dev, pk, round(frac * link_payload_gbps, 1), "host")
        r["offered_fraction_of_link"] = frac
        rows.append(r)
    rows.append(run_serving(xe, torch, dev, pk, 819.2, "host"))
    rows.append(run_serving(xe, torch, dev, pk, 819.2, "device"))
    rows.append(run_serving(xe, torch, dev, pk, None, "device"))
    del pk
    torch.cuda.empty_cache()
    return {"workload": "8 streams x 128 ch, N=256, T=4096 (8 frames per stream), Poisson arrivals, 0.1% drops, "
                        "0.5% reorders -> xe_stream_* (index + batched correlation + normalise per round)",
            "host_link_gbs": link, "runs": rows}


def workload_config(args):
    G = args.frames_per_call
    return {"workload": f"full band batched: N={N_INPUTS}, F={N_CHAN} channels, {args.frames} frames x "
                        f"T={N_TIME} from 16-byte-header UDP packets (128 streams x 8 ch, 0.1% lost), "
                        f"zero-copy assemble + correlate (accumulate), {G} consecutive frame(s) per call "
                        f"(T = {G * N_TIME} samples), normalise per integration",
            "n_inputs": N_INPUTS, "n_chan": N_CHAN, "n_time": N_TIME, "frames": args.frames,
            "frames_per_call": G,
            "l2": "inputs larger than L2 (distinct packets per frame)",
            "parallelism": (f"channel shards x{args.gpus}: rank r correlates channels [1024 r, 1024 r + 1024) of a "
                            f"{1024 * args.gpus}-channel band from its own packets; no collective on the data path")}


# ----------------------------------------------------------------------------- GPU arm

def make_packets(frames: int, device, seed: int = 3000, p_drop: float = 0.001, frames_per_group: int = 1):
    """64 distinct frames of synthetic packets, generated on the device (torch RNG), 0.1% dropped.
    Returns per-frame views [n_k][stride] and their counts; the frames of each group of
    frames_per_group consecutive frames lie back to back in one buffer, so that a group is also one
    contiguous packet array (one call over T = frames_per_group x 4096 samples)."""
    import torch

    import synth

    pkts, counts = [], []
    group = []
    for k in range(frames):
        fr = synth.signal_frame_torch(N_INPUTS, N_CHAN, N_TIME, seed + k, device=device, chunk=128)
        pk = synth.packetize_torch(fr, k * N_TIME // 4, GROUPS_PER_STREAM)
        del fr
        g = torch.Generator(device=device)
        g.manual_seed(seed + 7 * k)
        keep = torch.rand(pk.shape[0], generator=g, device=device) >= p_drop
        pk = pk[keep].contiguous()
        group.append(pk)
        counts.append(pk.shape[0])
        if len(group) == frames_per_group or k == frames - 1:
            buf = torch.cat(group) if len(group) > 1 else group[0]
            group.clear()
            off = 0
            for c in counts[len(pkts):]:
                pkts.append(buf[off:off + c])
                off += c
    return pkts, counts


def run_xe(args):
    import torch

    import paper_1503_06189_b300 as xe

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    N, F, T, FR, G = N_INPUTS, N_CHAN, N_TIME, args.frames, args.frames_per_call
    if G < 1 or FR % G or G * T > 1 << 15:
        raise SystemExit("--frames-per-call must divide --frames, with frames_per_call x 4096 <= 32768")
    pkts, counts = make_packets(FR, dev, seed=3000 + 100000 * rank, frames_per_group=G)
    stride = pkts[0].shape[1]
    filled = torch.empty((G * T // 4, F // 8), dtype=torch.uint8, device=dev)
    lost = torch.zeros(F, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.int32, device=dev)
    vis = torch.empty((F, npairs(N), 2), dtype=torch.int32, device=dev)
    out = torch.empty((F, npairs(N), 2), dtype=torch.float32, device=dev)
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(xe.Shape(N, F, G * T)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    n_ev = FR * max(args.steps, 1)
    ev_c0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ev_c1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]

    def calls(g):
        """(packet view, count, seq0) of each call when g consecutive frames go into one call: the
        frames of a call are contiguous in memory (groups of G, g dividing G)."""
        out_ = []
        for c in range(FR // g):
            k0 = c * g
            first = pkts[k0]
            n = sum(counts[k0:k0 + g])
            out_.append((first.as_strided((n, stride), (stride, 1)), n, k0 * T // 4))
        return out_

    def make_step(g):
        cl = calls(g)
        sg = xe.Shape(N, F, g * T)

        def step(ev_base=None):
            with torch.cuda.stream(stream):
                lost.zero_()
            for c, (pk, n, seq0) in enumerate(cl):
                if ev_base is not None:
                    ev_c0[ev_base + c].record(stream)
                xe.xe_correlate_packets(pk, n, stride, seq0, GROUPS_PER_STREAM, sg, vis, c > 0, filled, lost,
                                        stats, ws, stream=stream)
                if ev_base is not None:
                    ev_c1[ev_base + c].record(stream)
            xe.xe_normalize(vis, xe.Shape(N, F, FR * T), FR * T, lost, out, stream=stream)
        return step, len(cl)

    # the autotuner picks the pair engine's layout and launch shape for the calls this run makes
    from paper_1503_06189_b300 import autotune
    table = autotune.Table(args.tune_cache)
    table.tune_packets(N, G * T)
    if G > 1:
        table.tune_packets(N, T)
    table.install()
    tuning = [{k: e[k] for k in ("n_inputs", "t_bucket", "mode", "layout", "pairs", "odd_pairs", "k_flush", "ms")}
              for e in table.entries.values()]
    print(f"[bench] tuning {tuning}", file=sys.stderr, flush=True)

    step, n_calls = make_step(G)
    launches_per_step = n_calls * 4 + 1           # per call: init, claim, tally, correlation; + normalise

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            step(ev_base=k * n_calls)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    corr_ms = [ev_c0[k].elapsed_time(ev_c1[k]) for k in range(n_calls * args.steps)]
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clocks = clk.summary()
    print(f"[bench] device: {ms:.3f} ms/step, correlate {statistics.mean(corr_ms):.4f} ms/launch, clocks {clocks}",
          file=sys.stderr, flush=True)

    # the same step captured once into a CUDA graph and replayed (launch overhead amortised)
    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        with torch.cuda.stream(stream):          # replay on the stream the events are recorded on
            g.replay()
        torch.cuda.synchronize(dev)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            r0.record(stream)
            for _ in range(args.steps):
                g.replay()
            r1.record(stream)
        torch.cuda.synchronize(dev)
        graph_ms = r0.elapsed_time(r1) / args.steps
        del g
    except Exception as exc:  # capture is optional for the metric; report why it failed
        print(f"[bench] graph capture failed: {exc}", file=sys.stderr)

    # the same integration with one call per frame (T = 4096 per call), for comparison
    per_frame = None
    if G > 1:
        step1, n1 = make_step(1)
        for _ in range(args.warmup):
            step1()
        torch.cuda.synchronize(dev)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for k in range(args.steps):
            step1(ev_base=k * n1)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        ms1 = q0.elapsed_time(q1) / args.steps
        c1 = statistics.mean(ev_c0[k].elapsed_time(ev_c1[k]) for k in range(n1 * args.steps))
        per_frame = {"ms_per_step": ms1, "value": cmac_per_frame() * FR / (ms1 / 1e3) * world, "unit": "CMAC/s",
                     "correlate_ms_per_call": c1, "frames_per_call": 1}
        print(f"[bench] one call per frame: {ms1:.3f} ms/step, correlate {c1:.4f} ms/launch", file=sys.stderr,
              flush=True)

    baselines = run_engine_baselines(xe, torch, dev)

    # end to end through host buffers: pinned packets -> H2D per call -> same calls -> D2H of result
    e2e = run_e2e(xe, torch, dev, pkts, counts, stride, args)
    del pkts
    torch.cuda.empty_cache()
    serving = None
    if not args.no_serving:
        try:
            serving = run_serving_suite(xe, torch, dev)
        except Exception as exc:
            serving = {"error": str(exc)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cmac_step = cmac_per_frame() * FR
    value = cmac_step / (ms / 1e3) * world
    pk, how = peaks()
    peak_tflops = 2.0 * pk["bf16_tflops_sustained"]      # FP8 dense = 2 x bf16 (nominal ratio)
    corr_avg_ms = statistics.mean(corr_ms)
    achieved = cmac_per_frame() * G * 8 / (corr_avg_ms / 1e3) / 1e12
    traffic = load_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "CMAC/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp8 (e4m3 x e4m3, e5m2 x e5m2) -> f32 (exact int), int32 out", "data": "synthetic",
        "config": workload_config(args),
        "realtime_factor": FR * T / SAMPLE_RATE / (ms / 1e3),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "peak_burst": 2.0 * pk["bf16_tflops"], "frac_burst": achieved / (2.0 * pk["bf16_tflops"]),
                     "kernel": f"xe_correlate_packets over {G} frame(s) per call (index kernels + packet-mode "
                               "CTA-pair tcgen05 correlation), 8 int ops per CMAC, timed by CUDA events around each call",
                     "peak_source": f"{how}: 2 x bf16_tflops_sustained (FP8 kind::f8f6f4 dense)"},
        "gpu_launches": launches_per_step * args.steps,
        "tuning": tuning,
        "graph_ms_per_step": graph_ms,
        "one_call_per_frame": per_frame,
        "engine_baselines": baselines,
        "clocks": clocks,
        "e2e": e2e,
        "serving": serving,
    }
    if world == 1 or rank == 0:
        line["cpu_baseline"] = {k: v for k, v in cpu_oracle_sample().items() if k != "seconds"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_engine_baselines(xe, torch, dev, reps: int = 3):
    """The legacy warp-level engines (mma.sync m16n8k64 s4 on the packed samples, m16n8k32 s8 on
    samples unpacked in shared memory) and the default CTA-pair tcgen05 engine on the same assembled
    full-band frame (N=256, F=1024, T=4096, random
    bytes), best of `reps` launches each: context for what the tensor-core path buys."""
    N, F, T = N_INPUTS, N_CHAN, N_TIME
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    frame = torch.randint(0, 256, (T, F, N), generator=g, device=dev, dtype=torch.int32).to(torch.uint8)
    vis = torch.empty((F, npairs(N), 2), dtype=torch.int32, device=dev)
    out = {}
    for name, eng in (("legacy_mma_sync_s4", xe.XE_ENGINE_LEGACY_S4), ("legacy_mma_sync_s8", xe.XE_ENGINE_LEGACY_S8),
                      ("tcgen05_pair", xe.XE_ENGINE_FUSED_PAIR)):
        tune = dict(engine=eng, max_strip=0, k_flush=0, n_ctas=0)
        jobs = [(frame, vis, xe.Shape(N, F, T), False)]
        ws = torch.empty(max(1, xe.xe_correlate_batched_workspace_size(jobs, tune)), dtype=torch.uint8, device=dev)
        best = None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            xe.xe_correlate_batched(jobs, ws, tune)
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = {"ms_per_frame": best, "value": cmac_per_frame() / (best / 1e3), "unit": "CMAC/s"}
        del ws
    out["per_channel_launches"] = run_per_channel_launches(xe, torch, dev, frame, vis, reps)
    del frame, vis
    torch.cuda.empty_cache()
    out["workload"] = "one assembled full-band frame, N=256, F=1024, T=4096, random bytes, xe_correlate_batched"
    return out


def run_per_channel_launches(xe, torch, dev, frame, vis, reps: int = 3):
    """The plain form of the same correlation: one xe_correlate launch per channel (F = 1), each on
    that channel's samples copied to a contiguous [T][1][N] frame before timing, issued one after
    the other on one stream; also replayed from a CUDA graph holding those launches (no host launch
    cost). `vis` holds the batched launch's result (the last engine run above, on the same frame);
    both forms must reproduce it bit for bit."""
    N, F, T = N_INPUTS, N_CHAN, N_TIME
    s1 = xe.Shape(N, 1, T)
    per = frame.permute(1, 0, 2).contiguous()               # [F][T][N] = F frames of [T][1][N]
    got = torch.full_like(vis, -1)
    ws = torch.empty(max(1, xe.xe_correlate_workspace_size(s1)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def launches():
        for f in range(F):
            xe.xe_correlate(per[f], s1, got[f], False, ws, stream=stream)

    def timed(fn):
        best = None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    with torch.cuda.stream(stream):
        plain_ms = timed(launches)
        identical = bool(torch.equal(got, vis))
        got.fill_(-1)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            launches()
        graph_ms = timed(graph.replay)
        identical = identical and bool(torch.equal(got, vis))
    del graph, per, got, ws
    torch.cuda.empty_cache()
    return {"launches": F, "ms_per_frame": plain_ms, "value": cmac_per_frame() / (plain_ms / 1e3),
            "graph_ms_per_frame": graph_ms, "graph_value": cmac_per_frame() / (graph_ms / 1e3),
            "unit": "CMAC/s", "identical_to_batched": identical}


def load_traffic():
    """DRAM bytes per correlation launch from the committed ncu summary, or None when the kernel
    source has changed since those counters were taken."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    src = os.path.join(ROOT, d.get("source", ""))
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != d.get("source_sha256_16"):
        return None
    return d.get("correlate_bytes_per_launch")


def run_e2e(xe, torch, dev, pkts, counts, stride, args):
    """Same integration through host buffers: the packets of G consecutive frames (one call) sit in
    pinned host memory; every call copies them to the device on a copy stream, double-buffered
    against compute, and correlates them (each call re-integrates those frames, sequence numbers
    as in the packets); the normalised matrix is copied back at the end of every step."""
    N, F, T, FR, G = N_INPUTS, N_CHAN, N_TIME, args.frames, args.frames_per_call
    sg = xe.Shape(N, F, G * T)
    n = sum(counts[:G])
    ring = pkts[0].as_strided((n, stride), (stride, 1)).cpu().pin_memory()
    dbuf = [torch.empty((n, stride), dtype=torch.uint8, device=dev) for _ in range(2)]
    filled = torch.empty((G * T // 4, F // 8), dtype=torch.uint8, device=dev)
    lost = torch.zeros(F, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.int32, device=dev)
    vis = torch.empty((F, npairs(N), 2), dtype=torch.int32, device=dev)
    out = torch.empty((F, npairs(N), 2), dtype=torch.float32, device=dev)
    host_out = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(sg), dtype=torch.uint8, device=dev)
    comp = torch.cuda.Stream(device=dev)
    copy = torch.cuda.Stream(device=dev)
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def one_step():
        with torch.cuda.stream(comp):
            lost.zero_()
        for c in range(FR // G):
            b = c % 2
            with torch.cuda.stream(copy):
                copy.wait_event(used[b])
                dbuf[b].copy_(ring, non_blocking=True)
                h2d_done[b].record(copy)
            comp.wait_event(h2d_done[b])
            xe.xe_correlate_packets(dbuf[b], n, stride, 0, GROUPS_PER_STREAM, sg, vis, c > 0, filled, lost, stats, ws,
                                    stream=comp)
            used[b].record(comp)
        xe.xe_normalize(vis, xe.Shape(N, F, FR * T), FR * T, lost, out, stream=comp)
        with torch.cuda.stream(comp):
            host_out.copy_(out, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        one_step()
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
        comp.synchronize()
    dt = (time.perf_counter() - t0) / steps
    h2d = ring.numel() * (FR // G)
    return {"value": cmac_per_frame() * FR / dt, "unit": "CMAC/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(out.numel() * 4), "ms_per_step": dt * 1e3,
            "realtime_factor": FR * T / SAMPLE_RATE / dt, "frames_per_call": G,
            "note": "every call copies its packets (G frames) from pinned host memory inside the timed region; "
                    "one call's packet set is re-sent for each call of the step (the same bytes, real transfers)"}


# ----------------------------------------------------------------------------- configurations 1, 2, 4

def config_shapes(cfg):
    if cfg == 1:
        return [(16, 4, 4096)]
    if cfg == 2:
        return [(256, 64, 16384)]
    if cfg == 6:
        return [(2048, 64, 16384)]
    import synth
    return synth.config4_shapes()


def config_workload(cfg):
    return {1: "tiny: N=16, F=4, T=4096, uniform 4+4-bit nibbles (seed 1); correlate + normalise",
            2: "Pathfinder per-server frame: N=256, F=64, T=16384 (256 MiB), signal model (seed 2); "
               "correlate + normalise",
            4: "uneven batch: 24 jobs (seed 4), N 64..2048, F 16..256, T 1024..32768 (27.6 GiB of frames), "
               "one batched correlation launch + per-job normalise",
            6: "full-CHIME scale per server: N=2048, F=64, T=16384 (2 GiB), signal model (seed 6); "
               "correlate + normalise"}[cfg]


def config_frame_host(cfg, k, N, F, T):
    import synth
    if cfg == 1:
        return synth.uniform_frame(N, F, T, 1)
    return synth.signal_frame(N, F, T, {2: 2, 6: 6}.get(cfg, 4000 + k))


def run_config_reference(args):
    """The oracle on configuration 1 or 2 in full, or on a bounded sample of configuration 4 (first
    channel of the jobs, smallest first, until about 10 s of CPU work)."""
    import oracle

    cfg = args.config
    shapes = config_shapes(cfg)
    cmac, dt, done = 0, 0.0, []
    order = sorted(range(len(shapes)), key=lambda k: shapes[k][0] ** 2 * shapes[k][2])
    for k in order:
        N, F, T = shapes[k]
        chans = F if cfg in (1, 2) else 1
        fr = config_frame_host(cfg, k, N, chans, T)
        reps = 0
        while reps == 0 or (cfg == 1 and dt < 2.0):        # the tiny frame: repeat for ~2 s
            ts = time.perf_counter()
            v, st = oracle.correlate(fr, 0, chans)
            n = oracle.counts_from_counters(T, [0] * chans, N)
            oracle.normalize(v, n)
            dt += time.perf_counter() - ts
            cmac += chans * npairs(N) * T
            reps += 1
        done.append(f"{chans} ch of N={N}, T={T}" + (f" x{reps}" if reps > 1 else ""))
        if cfg != 4 or dt >= 10.0:
            break
    return {"value": cmac / dt, "unit": "CMAC/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": ("full configuration: " if cfg in (1, 2) else "bounded sample: ") + "; ".join(done)
                      + f" ({dt:.1f} s of CPU work)", "seconds": dt}


def block_products(N, layout):
    """256 x 256 block products per sample and channel that the pair engine issues for N inputs:
    every Gram block on or above the block diagonal, or with the fold layout two per whole
    256-input super-block plus the Gram blocks outside the super-blocks."""
    import paper_1503_06189_b300 as xe

    nb = -(-2 * N // 256)
    fold = nb >= 2 and layout in (xe.XE_LAYOUT_AUTO, xe.XE_LAYOUT_FOLD)
    if not fold:
        return nb * (nb + 1) // 2
    return 2 * (nb // 2) + (nb & 1) + sum(max(0, nb - 2 * (r // 2 + 1)) for r in range(nb))


def useful_mma_fraction(shapes, layouts=None):
    """Useful real MACs (4 per CMAC) over the MMA work the pair engine issues (block_products per
    job; `layouts` per job, default: whole Gram blocks). Above 1 where the fold layout's two
    products cover a super-block's Hermitian square."""
    import paper_1503_06189_b300 as xe

    useful = issued = 0
    for k, (N, F, T) in enumerate(shapes):
        lay = layouts[k] if layouts else xe.XE_LAYOUT_FRAME_BLOCKS
        useful += 4 * npairs(N) * F * T
        issued += block_products(N, lay) * 256 * 256 * F * T
    return useful / issued


def run_config(args):
    import torch

    import paper_1503_06189_b300 as xe
    import synth

    cfg = args.config
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = config_shapes(cfg)
    frames, vis, outs, lost = [], [], [], []
    for k, (N, F, T) in enumerate(shapes):
        if cfg == 1:
            fr = torch.from_numpy(config_frame_host(cfg, k, N, F, T)).to(dev)
        else:
            fr = synth.signal_frame_torch(N, F, T, {2: 2, 6: 6}.get(cfg, 4000 + k), device=dev,
                                          chunk=max(1, (1 << 27) // (T * N)))
        frames.append(fr)
        vis.append(torch.empty((F, npairs(N), 2), dtype=torch.int32, device=dev))
        outs.append(torch.empty((F, npairs(N), 2), dtype=torch.float32, device=dev))
        lost.append(torch.zeros(F, dtype=torch.int32, device=dev))
    jobs = [(fr, v, xe.Shape(*sh), False) for fr, v, sh in zip(frames, vis, shapes)]
    ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    # the autotuner picks the pair engine's kernel, layout and launch shape per (N, T-bucket) of the jobs
    from paper_1503_06189_b300 import autotune
    table = autotune.Table(args.tune_cache)
    for N, F, T in shapes:
        table.tune_frames(N, T)
    table.install()
    tuning = [{k: e[k] for k in ("n_inputs", "t_bucket", "mode", "layout", "pairs", "odd_pairs", "ms")}
              for e in table.entries.values()]
    # the layout each job runs: the largest job's entry picks the kernel for the whole launch
    layouts = [table.entries[autotune.key("frames", N, T)]["layout"] for N, F, T in shapes]
    big_n, _, big_t = max(shapes, key=lambda sh: sh[1] * npairs(sh[0]) * sh[2])
    if any(T % 4 for N, F, T in shapes) or \
            table.entries[autotune.key("frames", big_n, big_t)]["layout"] == xe.XE_LAYOUT_FRAME_BLOCKS:
        layouts = [xe.XE_LAYOUT_FRAME_BLOCKS] * len(shapes)      # the 256-sample kernel
    else:
        layouts = [xe.XE_LAYOUT_AUTO if lay == xe.XE_LAYOUT_FRAME_BLOCKS else lay for lay in layouts]
    reps = {1: 2000, 2: 20, 4: 1, 6: 2}[cfg]           # launches per step: a step lasts >= ~10 ms
    cmac_step = reps * sum(F * npairs(N) * T for N, F, T in shapes)
    n_ev = reps * max(args.steps, 1)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]

    def step(base=None):
        for r in range(reps):
            if base is not None:
                ev0[base + r].record(stream)
            xe.xe_correlate_batched(jobs, ws, stream=stream)
            if base is not None:
                ev1[base + r].record(stream)
            for (N, F, T), v, o, l in zip(shapes, vis, outs, lost):
                xe.xe_normalize(v, xe.Shape(N, F, T), T, l, o, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MiB > L2, between steps
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms_total = 0.0
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            e0.record(stream)
            step(base=k * reps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_total += e0.elapsed_time(e1)
    ms = ms_total / args.steps
    corr_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    clocks = clk.summary()

    # the same step captured once into a CUDA graph and replayed
    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize(dev)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gms = 0.0
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                r0.record(stream)
                g.replay()
                r1.record(stream)
            torch.cuda.synchronize(dev)
            gms += r0.elapsed_time(r1)
        graph_ms = gms / args.steps
        del g
    except Exception as exc:
        print(f"[bench] graph capture failed: {exc}", file=sys.stderr)

    # end to end: frames from pinned host memory, correlate + normalise, results back
    e2e = None
    try:
        hosts = [fr.cpu().pin_memory() for fr in frames]
        host_out = [torch.empty(o.shape, dtype=torch.float32).pin_memory() for o in outs]
        for _ in range(2):
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                for h, fr in zip(hosts, frames):
                    fr.copy_(h, non_blocking=True)
            step()
            with torch.cuda.stream(stream):
                for h, o in zip(host_out, outs):
                    h.copy_(o, non_blocking=True)
            stream.synchronize()
            dt = time.perf_counter() - t0
        e2e = {"value": cmac_step / dt, "unit": "CMAC/s", "h2d_bytes_per_step": int(sum(h.numel() for h in hosts)),
               "d2h_bytes_per_step": int(sum(o.numel() * 4 for o in outs)), "ms_per_step": dt * 1e3}
        del hosts, host_out
    except Exception as exc:
        e2e = {"error": str(exc)}

    if rank != 0:
        return 0
    pk, how = peaks()
    peak_tflops = 2.0 * pk["bf16_tflops_sustained"]
    achieved = cmac_step / reps * 8 / (corr_ms / 1e3) / 1e12
    sky = {1: 4096, 2: 16384, 6: 16384}.get(cfg)
    line = {
        "metric": METRIC, "value": cmac_step / (ms / 1e3), "unit": "CMAC/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp8 (e4m3 x e4m3, e5m2 x e5m2) -> f32 (exact int), int32 out", "data": "synthetic",
        "config": {"workload": config_workload(cfg), "config": cfg, "launches_per_step": reps,
                   "l2": "256 MiB written between steps" + ("; the tiny frame itself fits in L2" if cfg == 1 else "")},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None,
                     "peak_burst": 2.0 * pk["bf16_tflops"], "frac_burst": achieved / (2.0 * pk["bf16_tflops"]),
                     "useful_mma_fraction": useful_mma_fraction(shapes, layouts),
                     "kernel": "xe_correlate_batched (CTA-pair tcgen05 correlation), 8 int ops per CMAC",
                     "peak_source": f"{how}: 2 x bf16_tflops_sustained (FP8 kind::f8f6f4 dense)"},
        "gpu_launches": args.steps * reps * (1 + len(shapes)),
        "clocks": clocks, "e2e": e2e,
    }
    line["tuning"] = tuning
    line["graph_ms_per_step"] = graph_ms
    if sky:
        line["realtime_factor"] = cmac_step / (ms / 1e3) / (npairs(shapes[0][0]) * shapes[0][1] * SAMPLE_RATE)
    base = run_config_reference(args)
    line["cpu_baseline"] = {k: v for k, v in base.items() if k != "seconds"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--frames", type=int, default=N_FRAMES)
    ap.add_argument("--frames-per-call", type=int, default=8,
                    help="consecutive frames correlated by one call (T = 4096 x this <= 32768: the accumulator "
                         "stays in tensor memory across them)")
    ap.add_argument("--impl", choices=["xe", "reference"], default="xe")
    ap.add_argument("--no-serving", action="store_true", help="skip the configuration-5 serving run")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of the autotuner's entries: read if it exists, written after tuning (a profiled "
                         "run then launches what the plain run chose)")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 6], default=3,
                    help="3: the full-band integration (default); 1, 2, 4: the other workloads; 6: N=2048 per server")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.config != 3:
            if int(os.environ.get("RANK", "0")) != 0:
                return 0
            base = run_config_reference(args)
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "CMAC/s",
                              "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": base["seconds"] * 1e3,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                              "data": "synthetic", "config": {"workload": config_workload(args.config)},
                              "cpu_baseline": {k: v for k, v in base.items() if k != "seconds"},
                              "e2e": {"value": base["value"], "unit": "CMAC/s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}), flush=True)
            return 0
        return run_reference(args)
    if args.config != 3:
        return run_config(args)
    return run_xe(args)


if __name__ == "__main__":
    sys.exit(main())
