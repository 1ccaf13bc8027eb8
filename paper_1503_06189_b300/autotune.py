"""Autotuner for the correlation's work-item shape per (N, T-bucket): the single-CTA fused engine's
strip width (1..4 tiles of 128x128 along one row of the Gram matrix per work item), and whether the
CTA-pair engine (256x256 blocks) beats it.

Wider strips reuse each converted operand block across more tiles and save conversions; narrower
strips double-buffer the tensor-memory accumulator and spread small problems over more SMs. The best
choice depends on N (how many tiles a channel has) and T (how long each work item runs), so it is
measured: each candidate runs on a seeded random frame of the bucket's shape on the device, timed
with CUDA events (best of `reps`), and the winner is cached in a JSON file keyed "N<N>_T<bucket>".

    table = autotune.Table(path)               # loads the cache if the file exists
    ms = table.best(N, T)                      # tunes on first use, then reads the cache
    jobs = [(frame, vis, shape, acc, table.best(shape.n_inputs, shape.n_time)) ...]
"""
from __future__ import annotations

import json
import os

import torch

import paper_1503_06189_b300 as xe

CANDIDATES = (1, 2, 3, 4)
PROBE_BYTES = 256 << 20          # frame bytes of one probe launch
PROBE_ITEMS = 4 * 148            # aim for about four waves of work items


def bucket(n_time: int) -> int:
    """Power of two >= T (at least 128): T values in one bucket share a tuning."""
    return 1 << max(7, (max(int(n_time), 1) - 1).bit_length())


def key(n_inputs: int, n_time: int) -> str:
    return f"N{int(n_inputs)}_T{bucket(n_time)}"


def _strips(n_inputs: int, ms: int) -> int:
    nb = -(-2 * n_inputs // 128)
    total = 0
    for rb in range(nb):
        wd = min(ms, nb - rb)
        wo = min(ms, 3)
        total += 1 + -(-(nb - rb - wd) // wo)
    return total


def measure(n_inputs: int, n_time: int, candidates=CANDIDATES, reps: int = 3, device=None) -> dict:
    """Milliseconds per launch for each candidate strip width on a probe frame of this bucket."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    T = bucket(n_time)
    per_chan = T * n_inputs
    F = max(1, min(PROBE_BYTES // per_chan, -(-PROBE_ITEMS // _strips(n_inputs, max(candidates)))))
    g = torch.Generator(device=dev)
    g.manual_seed(n_inputs * 131 + T)
    frame = torch.randint(0, 256, (T, F, n_inputs), generator=g, device=dev, dtype=torch.int32).to(torch.uint8)
    s = xe.Shape(n_inputs, F, T)
    vis = torch.empty((F, xe.npairs(n_inputs), 2), dtype=torch.int32, device=dev)
    out = {}
    for ms in list(candidates) + ["pair"]:
        pair = ms == "pair"
        jobs = [(frame, vis, s, False, 0 if pair else ms)]
        tune = dict(engine=xe.XE_ENGINE_FUSED_PAIR if pair else xe.XE_ENGINE_FUSED, max_strip=0 if pair else ms,
                    k_flush=0, n_ctas=0)
        ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs, tune), dtype=torch.uint8, device=dev)
        xe.xe_correlate_batched(jobs, ws, tune)                       # warm-up
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            xe.xe_correlate_batched(jobs, ws, tune)
            e1.record()
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        out[ms] = best
    return out


class Table:
    """Cached strip widths per (N, T-bucket), persisted as JSON at `path` (None: in memory only)."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries: dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def _entry(self, n_inputs: int, n_time: int) -> dict:
        k = key(n_inputs, n_time)
        if k not in self.entries:
            ms = measure(n_inputs, n_time)
            strips = {c: v for c, v in ms.items() if c != "pair"}
            win = min(strips, key=strips.get)
            self.entries[k] = {"max_strip": int(win), "pair_wins": bool(ms["pair"] < strips[win]),
                               "ms": {str(c): round(v, 4) for c, v in ms.items()}}
            self.save()
        return self.entries[k]

    def best(self, n_inputs: int, n_time: int) -> int:
        """Best strip width of the single-CTA fused engine for this bucket."""
        return int(self._entry(n_inputs, n_time)["max_strip"])

    def best_engine(self, n_inputs: int, n_time: int) -> int:
        """XE_ENGINE_FUSED_PAIR if the CTA-pair engine beat every strip width, else XE_ENGINE_FUSED."""
        return xe.XE_ENGINE_FUSED_PAIR if self._entry(n_inputs, n_time)["pair_wins"] else xe.XE_ENGINE_FUSED

    def save(self):
        if not self.path:
            return
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)
