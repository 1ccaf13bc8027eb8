"""Small, self-contained workloads for profiling one libxe kernel at a time (ncu captures).

    python -m paper_1503_06189_b300.prof correlate --n 256 --f 128 --t 4096 --iters 3 [--engine 1]
    python -m paper_1503_06189_b300.prof assemble  --n 256 --f 128 --t 4096 --iters 3
    python -m paper_1503_06189_b300.prof normalize --n 256 --f 128 --iters 3
    python -m paper_1503_06189_b300.prof packets   --n 256 --f 128 --t 4096 --iters 3
    python -m paper_1503_06189_b300.prof flags     --n 256 --f 256 --t 4096 --iters 3
    python -m paper_1503_06189_b300.prof shift     --n 256 --f 128 --t 4096 --iters 3 [--spread 64] [--uniform]

Inputs are uniform random bytes generated on the device; sizes default to a frame larger than L2
(128 MiB) so that DRAM counters are meaningful, while the device footprint stays at a few GB.
"""
from __future__ import annotations

import argparse
import sys
import time

import torch

import paper_1503_06189_b300 as xe


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["correlate", "assemble", "normalize", "packets", "flags", "mma_legacy",
                                       "shift"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--f", type=int, default=128)
    ap.add_argument("--t", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--engine", type=int, default=0)
    ap.add_argument("--max-strip", type=int, default=0)
    ap.add_argument("--accumulate", action="store_true", help="correlate, packets: add into the visibilities, as an integration does")
    ap.add_argument("--order", choices=["arrival", "group"], default="arrival",
                    help="packets: keep arrival (sequence-major) order or sort them group-major")
    ap.add_argument("--align", action="store_true",
                    help="packets: re-lay the packets at a 128-byte multiple stride with 128-byte aligned payloads")
    ap.add_argument("--zero-copy-only", action="store_true",
                    help="packets: time xe_correlate_packets only (no assembled frame is allocated)")
    ap.add_argument("--shift-max", type=int, default=-1,
                    help="packets: read the samples time-shifted (one delay per 16 inputs, 0 .. this many "
                         "samples) with xe_correlate_packets_shifted; the two-step path then shifts the frame")
    ap.add_argument("--spread", type=int, default=64, help="shift: delays drawn from 0 .. spread samples")
    ap.add_argument("--uniform", action="store_true", help="shift: one delay per block of 16 inputs")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    N, F, T = a.n, a.f, a.t
    s = xe.Shape(N, F, T)
    P = xe.npairs(N)
    frame = torch.randint(0, 256, (T, F, N), generator=g, device=dev, dtype=torch.int32).to(torch.uint8)
    vis = torch.zeros((F, P, 2), dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    if a.op == "correlate":
        tune = dict(engine=a.engine, max_strip=a.max_strip, k_flush=0, n_ctas=0)
        jobs = [(frame, vis, s, a.accumulate)]
        ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs, tune), dtype=torch.uint8, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.iters)]
        for e0, e1 in evs:
            e0.record()
            xe.xe_correlate_batched(jobs, ws, tune)
            e1.record()
        torch.cuda.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        best = min(ms[1:] if len(ms) > 1 else ms)
        cmac = F * P * T
        print(f"correlate engine={a.engine} max_strip={a.max_strip} N={N} F={F} T={T}: best {best:.4f} ms, "
              f"{cmac / best / 1e9:.3f} TCMAC/s, {8 * cmac / best / 1e9:.1f} T int-op/s", flush=True)
    elif a.op == "assemble":
        import synth
        pk = synth.packetize_torch(frame, 0, 1)
        filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device=dev)
        lost = torch.zeros(F, dtype=torch.int32, device=dev)
        stats = torch.zeros(5, dtype=torch.int32, device=dev)
        out = torch.empty_like(frame)
        ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device=dev)
        for _ in range(a.iters):
            xe.xe_assemble(pk, pk.shape[0], pk.shape[1], 0, 1, s, out, filled, lost, stats, ws)
    elif a.op == "packets":
        # zero-copy assembly + correlation against assembly then correlation, same packets
        import synth
        pk = synth.packetize_torch(frame, 0, 1)
        del frame
        keep = torch.rand(pk.shape[0], generator=g, device=dev) >= 0.001
        pk = pk[keep].contiguous()
        del keep
        torch.cuda.empty_cache()                                # only the packets stay on the device
        if a.order == "group":                                  # all slots of a group together
            hdr = pk[:, :16].contiguous().view(torch.int32)
            key = (hdr[:, 0] & 0xFFFF).to(torch.int64) * (1 << 32) + hdr[:, 2].to(torch.int64)
            pk = pk[torch.argsort(key)].contiguous()
        if a.align:
            stride = (pk.shape[1] + 127) // 128 * 128
            buf = torch.zeros(pk.shape[0] * stride + 128, dtype=torch.uint8, device=dev)
            off = (112 - buf.data_ptr()) % 128                 # header at 112 mod 128: payload 128-aligned
            view = buf[off:off + pk.shape[0] * stride].view(pk.shape[0], stride)
            view[:, :pk.shape[1]] = pk
            pk = view
        filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device=dev)
        lost = torch.zeros(F, dtype=torch.int32, device=dev)
        stats = torch.zeros(5, dtype=torch.int32, device=dev)
        ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device=dev)
        if not a.zero_copy_only:
            out = torch.empty((T, F, N), dtype=torch.uint8, device=dev)
            wsa = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device=dev)
            wsc = torch.empty(xe.xe_correlate_workspace_size(s), dtype=torch.uint8, device=dev)

        import numpy as np
        delays = None
        if a.shift_max >= 0:
            rs = np.random.default_rng(5)
            delays = np.repeat(rs.integers(0, min(a.shift_max, T) + 1, N // 16), 16).astype(np.int32)
            if not a.zero_copy_only:
                shifted = torch.empty_like(out)

        def zero_copy():
            if delays is None:
                xe.xe_correlate_packets(pk, pk.shape[0], pk.shape[1], 0, 1, s, vis, a.accumulate, filled, lost, stats,
                                        ws)
            else:
                xe.xe_correlate_packets_shifted(pk, pk.shape[0], pk.shape[1], 0, 1, s, delays, vis, a.accumulate,
                                                filled, lost, stats, ws)

        def two_step():
            xe.xe_assemble(pk, pk.shape[0], pk.shape[1], 0, 1, s, out, filled, lost, stats, wsa)
            if delays is None:
                xe.xe_correlate(out, s, vis, a.accumulate, wsc)
            else:
                xe.xe_time_shift(out, s, delays, shifted)
                xe.xe_correlate(shifted, s, vis, a.accumulate, wsc)

        cmac = F * P * T
        runs = (("zero-copy", zero_copy),) + (() if a.zero_copy_only else (("two-step", two_step),))
        for name, fn in runs:
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.iters)]
            for e0, e1 in evs:
                e0.record()
                fn()
                e1.record()
            torch.cuda.synchronize()
            ms = [e0.elapsed_time(e1) for e0, e1 in evs]
            best = min(ms[1:] if len(ms) > 1 else ms)
            print(f"packets {name} N={N} F={F} T={T}: best {best:.4f} ms, {cmac / best / 1e9:.3f} TCMAC/s",
                  flush=True)
    elif a.op == "flags":
        # flag counts from packet footers: sparse flags, bursts and a few fully flagged samples
        import numpy as np

        import synth
        host = frame.cpu().numpy()
        del frame
        fl = synth.random_flags(T, F, N, 5, p_sample=0.001, p_burst=0.01, p_all=0.001)
        pk = torch.from_numpy(synth.packetize(host, 0, 1, fl)).to(dev)
        fc = torch.zeros((F, N), dtype=torch.int32, device=dev)
        fp = torch.zeros((F, P), dtype=torch.int32, device=dev)
        ws = torch.empty(xe.xe_flag_counts_workspace_size(s), dtype=torch.uint8, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.iters)]
        for e0, e1 in evs:
            e0.record()
            xe.xe_flag_counts(pk, pk.shape[0], pk.shape[1], 0, 1, s, fc, fp, ws)
            e1.record()
        torch.cuda.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        best = min(ms[1:] if len(ms) > 1 else ms)
        print(f"flags N={N} F={F} T={T}: best {best:.4f} ms for {pk.numel() / 1e6:.0f} MB of packets, "
              f"{float(np.mean(fl)) * 100:.3f}% of samples flagged", flush=True)
    elif a.op == "mma_legacy":
        # rates of the legacy warp-level integer tensor path (what the LEGACY engines run on) and of dp4a
        blocks = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
        sink = torch.empty(blocks * 256, dtype=torch.int32, device=dev)
        for kind, name, ops in ((0, "mma.sync m16n8k64 s4", 16384), (1, "mma.sync m16n8k32 s8", 8192),
                                (2, "dp4a s8 (CUDA cores)", 256)):
            iters = 4000 if kind < 2 else 40000
            xe.xe_probe_mma_legacy(kind, blocks, 10, sink)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            xe.xe_probe_mma_legacy(kind, blocks, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            total = blocks * 8 * iters * 8 * ops
            print(f"{name}: {total / ms / 1e9:.1f} T int-op/s ({blocks} CTAs x 8 warps x {iters} x 8 "
                  f"instructions in {ms:.3f} ms)", flush=True)
    elif a.op == "shift":
        # per-input sample delays (each input its own, or one per block of 16 inputs); 2 bytes per sample
        import numpy as np
        rng = np.random.default_rng(3)
        d = rng.integers(0, a.spread + 1, N // 16 if a.uniform else N)
        d = np.repeat(d, 16) if a.uniform else d
        out = torch.empty_like(frame)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.iters)]
        for e0, e1 in evs:
            e0.record()
            xe.xe_time_shift(frame, s, d, out)
            e1.record()
        torch.cuda.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        best = min(ms[1:] if len(ms) > 1 else ms)
        print(f"shift N={N} F={F} T={T} spread={a.spread} uniform={a.uniform}: best {best:.4f} ms, "
              f"{2 * frame.numel() / best / 1e6:.1f} GB/s", flush=True)
    else:
        lost = torch.zeros(F, dtype=torch.int32, device=dev)
        out = torch.empty((F, P, 2), dtype=torch.float32, device=dev)
        for _ in range(a.iters):
            xe.xe_normalize(vis, s, T, lost, out)
    torch.cuda.synchronize()
    print(f"{a.op} N={N} F={F} T={T} x{a.iters}: {(time.perf_counter() - t0) * 1e3:.1f} ms wall", file=sys.stderr)
    return 0


if __name__ == "__main__":
    sys.exit(main())
