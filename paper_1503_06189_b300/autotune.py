"""Autotuner of the CTA-pair engine, the engine every libxe correlation runs by default, per
(N, T-bucket) and mode. It fills libxe's tuning table (xe_tune_entry in include/xe.h):

- packet mode (xe_correlate_packets and the serving loop): the work-item layout -- fold items over
  whole 256-input super-blocks (whole, or with a channel's samples split evenly over the CTA pairs),
  Gram blocks with twins, or Gram blocks with wide singles -- and whether the launch takes an odd
  number of CTA pairs;
- frame mode (xe_correlate, xe_correlate_batched): the kernel and layout -- the 128-sample kernel
  (the packet-mode kernel reading the frame in 4-sample slots) with any of those layouts, or the
  256-sample frame kernel with every Gram block its own item -- the number of CTA pairs (fewer
  pairs can end a launch's last round of work items more evenly) and its parity.

Each candidate runs on seeded random samples of the bucket's shape on the device (F chosen so that
a launch has about four rounds of work items, within a few GB), timed with CUDA events (best of
`reps`); the winner is cached as JSON under "packets_N<N>_T<bucket>" or "frames_N<N>_T<bucket>" and
installed into libxe with xe_tune_table_set, after which every launch of that shape uses it.

    table = autotune.Table(path)          # loads the cache if the file exists
    table.tune_packets(256, 32768)        # measures on first use, then reads the cache
    table.tune_frames(2048, 16384)
    table.install()                       # xe_tune_table_set(all entries)
"""
from __future__ import annotations

import json
import os

import paper_1503_06189_b300 as xe

PAIRS = 74                      # CTA pairs resident on a B300 (one CTA per SM)
ROUNDS = 4                      # rounds of work items a probe launch aims for
PROBE_BYTES = 2 << 30           # samples of one probe launch at most
PACKET_FIELDS = ("layout", "odd_pairs")


def bucket(n_time: int) -> int:
    """Power of two >= T (at least 128): T values in one bucket share a tuning."""
    return 1 << max(7, (max(int(n_time), 1) - 1).bit_length())


def key(mode: str, n_inputs: int, n_time: int) -> str:
    return f"{mode}_N{int(n_inputs)}_T{bucket(n_time)}"


def blocks(n_inputs: int) -> int:
    """256-row blocks of the 2N-row Gram matrix (128 inputs each)."""
    return -(-2 * int(n_inputs) // 256)


def items_per_channel(n_inputs: int, layout: int, n_time: int) -> float:
    """Work items of one channel (the library's layouts; a twin counts half for each of its two
    channels)."""
    nb = blocks(n_inputs)
    if layout == xe.XE_LAYOUT_FRAME_BLOCKS:
        return nb * (nb + 1) / 2
    fold = nb >= 2 and layout in (xe.XE_LAYOUT_AUTO, xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_FOLD_SPLIT)
    if fold:
        return nb // 2 + (nb & 1) + sum(max(0, nb - 2 * (r // 2 + 1)) for r in range(nb))
    twin = layout == xe.XE_LAYOUT_GRAM_TWIN or (layout in (xe.XE_LAYOUT_AUTO, xe.XE_LAYOUT_GRAM)
                                                and n_time >= 16384)
    per_ch = (nb - 1) + (nb - 1) * (nb - 2) // 2
    return per_ch + (0.5 if twin else 1.0)


def row_layouts(n_inputs: int) -> list[int]:
    """Layouts of the 128-sample kernel worth measuring: fold or Gram blocks above 128 inputs (and
    the balanced split where a channel is one fold item), twins or wide singles for a single block."""
    nb = blocks(n_inputs)
    if nb == 1:
        return [xe.XE_LAYOUT_GRAM_TWIN, xe.XE_LAYOUT_GRAM_WIDE]
    return [xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_GRAM] + ([xe.XE_LAYOUT_FOLD_SPLIT] if nb == 2 else [])


def packet_candidates(n_inputs: int) -> list[dict]:
    """Layouts worth measuring in packet mode, each with and without an odd pair count."""
    return [dict(layout=lay, pairs=0, odd_pairs=odd, k_flush=0) for lay in row_layouts(n_inputs) for odd in (0, 1)]


def frame_candidates(n_inputs: int, n_chan: int, n_time: int = 4096) -> list[dict]:
    """Frame mode: the 128-sample kernel's layouts with and without an odd pair count (whole 4-sample
    slots only), and the 256-sample kernel with all pairs, an odd count, and the smallest count that
    keeps its number of rounds of work items (fewer pairs finish a ragged last round together)."""
    cands = []
    if n_time % 4 == 0:
        cands = [dict(layout=lay, pairs=0, odd_pairs=odd, k_flush=0) for lay in row_layouts(n_inputs)
                 for odd in (0, 1)]
    items = int(items_per_channel(n_inputs, xe.XE_LAYOUT_FRAME_BLOCKS, n_time)) * n_chan
    rounds = -(-items // PAIRS)
    even = -(-items // rounds)
    blk = dict(layout=xe.XE_LAYOUT_FRAME_BLOCKS, pairs=0, k_flush=0)
    cands += [dict(blk, odd_pairs=0), dict(blk, odd_pairs=1)]
    if even < PAIRS:
        cands.append(dict(blk, pairs=even, odd_pairs=0))
    return cands


def probe_chan(n_inputs: int, n_time: int, per_channel: float, multiple: int) -> int:
    """Channels of a probe launch: about ROUNDS rounds of work items within PROBE_BYTES."""
    f = max(1, round(ROUNDS * PAIRS / max(per_channel, 1e-9)))
    f = min(f, max(1, PROBE_BYTES // (n_time * n_inputs)))
    return max(multiple, f // multiple * multiple)


def _time(fn, reps: int) -> float:
    import torch

    fn()                                                           # warm-up
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def measure_packets(n_inputs: int, n_time: int, candidates=None, reps: int = 3) -> list[tuple[dict, float]]:
    """Milliseconds per xe_correlate_packets call for each candidate entry (zero-copy, accumulating)."""
    import torch

    import synth

    T = bucket(n_time)
    cands = candidates or packet_candidates(n_inputs)
    F = probe_chan(n_inputs, T, min(items_per_channel(n_inputs, c["layout"], T) for c in cands), 8)
    dev = torch.device("cuda", torch.cuda.current_device())
    frame = synth.uniform_frame_torch(n_inputs, F, T, n_inputs * 131 + T, device=dev)
    pk = synth.packetize_torch(frame, 0, 1)
    del frame
    s = xe.Shape(n_inputs, F, T)
    vis = torch.zeros((F, xe.npairs(n_inputs), 2), dtype=torch.int32, device=dev)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device=dev)
    lost = torch.zeros(F, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.int32, device=dev)
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device=dev)
    saved = xe.xe_tune_table_get()
    out = []
    try:
        for c in cands:
            xe.xe_tune_table_set([dict(c, n_inputs=n_inputs, t_bucket=T, mode=xe.XE_TUNE_PACKETS)])
            ms = _time(lambda: xe.xe_correlate_packets(pk, pk.shape[0], pk.shape[1], 0, 1, s, vis, True, filled, lost,
                                                       stats, ws), reps)
            out.append((c, ms))
    finally:
        xe.xe_tune_table_set(saved)
    return out


def measure_frames(n_inputs: int, n_time: int, candidates=None, reps: int = 3) -> list[tuple[dict, float]]:
    """Milliseconds per xe_correlate_batched launch (one job of the bucket's shape) per candidate."""
    import torch

    import synth

    T = bucket(n_time)
    F = probe_chan(n_inputs, T, items_per_channel(n_inputs, xe.XE_LAYOUT_AUTO, T), 1)    # fewest items
    cands = candidates or frame_candidates(n_inputs, F, T)
    dev = torch.device("cuda", torch.cuda.current_device())
    frame = synth.uniform_frame_torch(n_inputs, F, T, n_inputs * 137 + T, device=dev)
    vis = torch.zeros((F, xe.npairs(n_inputs), 2), dtype=torch.int32, device=dev)
    jobs = [(frame, vis, xe.Shape(n_inputs, F, T), False)]
    ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs), dtype=torch.uint8, device=dev)
    saved = xe.xe_tune_table_get()
    out = []
    try:
        for c in cands:
            xe.xe_tune_table_set([dict(c, n_inputs=n_inputs, t_bucket=T, mode=xe.XE_TUNE_FRAMES)])
            out.append((c, _time(lambda: xe.xe_correlate_batched(jobs, ws), reps)))
    finally:
        xe.xe_tune_table_set(saved)
    return out


class Table:
    """Tuned entries per (mode, N, T-bucket), persisted as JSON at `path` (None: in memory only)."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries: dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def _tune(self, mode: str, n_inputs: int, n_time: int) -> dict:
        k = key(mode, n_inputs, n_time)
        if k not in self.entries:
            res = (measure_packets if mode == "packets" else measure_frames)(n_inputs, n_time)
            best, best_ms = min(res, key=lambda r: r[1])
            self.entries[k] = {"n_inputs": int(n_inputs), "t_bucket": bucket(n_time),
                               "mode": xe.XE_TUNE_PACKETS if mode == "packets" else xe.XE_TUNE_FRAMES,
                               "layout": int(best["layout"]), "pairs": int(best["pairs"]),
                               "odd_pairs": int(best["odd_pairs"]), "k_flush": int(best["k_flush"]),
                               "ms": round(best_ms, 4),
                               "measured": [dict(c, ms=round(ms, 4)) for c, ms in res]}
            self.save()
        return self.entries[k]

    def tune_packets(self, n_inputs: int, n_time: int) -> dict:
        return self._tune("packets", n_inputs, n_time)

    def tune_frames(self, n_inputs: int, n_time: int) -> dict:
        return self._tune("frames", n_inputs, n_time)

    def c_entries(self) -> list[dict]:
        fields = ("n_inputs", "t_bucket", "mode", "layout", "pairs", "odd_pairs", "k_flush")
        return [{f: e[f] for f in fields} for e in self.entries.values()]

    def install(self):
        """Loads every entry into libxe's tuning table."""
        xe.xe_tune_table_set(self.c_entries())

    def save(self):
        if not self.path:
            return
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)
