"""Small, self-contained workloads for profiling one libxe kernel at a time (ncu captures).

    python -m paper_1503_06189_b300.prof correlate --n 256 --f 128 --t 4096 --iters 3 [--engine 1]
    python -m paper_1503_06189_b300.prof assemble  --n 256 --f 128 --t 4096 --iters 3
    python -m paper_1503_06189_b300.prof normalize --n 256 --f 128 --iters 3

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
    ap.add_argument("op", choices=["correlate", "assemble", "normalize"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--f", type=int, default=128)
    ap.add_argument("--t", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--engine", type=int, default=0)
    ap.add_argument("--max-strip", type=int, default=0)
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
        jobs = [(frame, vis, s, False)]
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
