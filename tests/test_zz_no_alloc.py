"""xe_assemble_noalloc against xe_assemble (GPU, through the C ABI).

The allocation-free entry point serves callers that cannot allocate device memory where they
assemble frames (non-blocking receive loops, or a host that owns all device memory); its scratch
is a fixed array inside the library that every call reuses. This file is
collected last on purpose, so that a run stopping at its first failure has run everything else. The
checks: two calls in a row on different packet sets must each give exactly what the workspace entry
point gives (assembly is integer work: bit-exact), the second call must not see leftovers of the
first, and frames above the static table's size must be refused.
"""
import numpy as np
import pytest
import torch

import synth
import paper_1503_06189_b300 as xe

pytestmark = pytest.mark.gpu


def _outputs(shape):
    T, F, N = shape.n_time, shape.n_chan, shape.n_inputs
    return (torch.full((T, F, N), 0xA5, dtype=torch.uint8, device="cuda"),
            torch.full((T // 4, F // 8), 7, dtype=torch.uint8, device="cuda"),
            torch.zeros(F, dtype=torch.int32, device="cuda"),
            torch.zeros(5, dtype=torch.int32, device="cuda"))


def test_noalloc_matches_workspace_entry_point_twice():
    N, F, T, gps = 256, 64, 512, 2
    s = xe.Shape(N, F, T)
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    for call, (seed, p_drop, p_dup) in enumerate([(101, 0.05, 0.02), (202, 0.30, 0.10)]):
        fr = synth.signal_frame(N, F, T + 32, seed)
        seq0 = 1000 + call * 500
        pk = synth.packet_stream(fr, seq0 - 4, gps, seed=seed + 1, p_drop=p_drop, p_reorder=0.05, p_dup=p_dup)
        pkd = torch.from_numpy(pk).cuda()
        ref = _outputs(s)
        got = _outputs(s)
        xe.xe_assemble(pkd, pk.shape[0], pk.shape[1], seq0, gps, s, *ref, ws)
        xe.xe_assemble_noalloc(pkd, pk.shape[0], pk.shape[1], seq0, gps, s, *got)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            assert torch.equal(r, g), f"call {call}: allocation-free result differs"
        assert int(got[3][0]) > 0 and int(got[3][2]) > 0           # ok and late packets both seen


def test_noalloc_rejects_frames_beyond_static_table():
    N = 16
    T = 4 * 2048
    F = 8 * (xe.XE_ASSEMBLE_NOALLOC_MAX_SLOTS // 2048 + 1)           # one group too many
    s = xe.Shape(N, F, T)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    counters = torch.zeros(max(F, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(xe.XeError) as e:
        xe.xe_assemble_noalloc(dummy, 0, 16 + 32 * N, 0, 1, s, dummy, dummy, counters, counters)
    assert e.value.status == xe.XE_ENOMEM
