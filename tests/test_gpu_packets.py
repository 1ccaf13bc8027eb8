"""Zero-copy assembly + correlation (xe_correlate_packets) through the C ABI (GPU).

The call must give exactly what the two-step path gives: the oracle's assembly of the packets
(Sec. II-A.2) followed by the oracle's correlation of that frame (Sec. II-B). Integer work, so every
comparison is bit-exact: vis, filled, lost and stats.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu


def _packets_gpu(pk, seq0, gps, N, F, T, vis=None, accumulate=False, lost=None, stats=None):
    s = xe.Shape(N, F, T)
    vis = torch.full((F, xe.npairs(N), 2), -12345, dtype=torch.int32, device="cuda") if vis is None else vis
    filled = torch.full((T // 4, F // 8), 7, dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda") if lost is None else lost
    stats = torch.zeros(5, dtype=torch.int32, device="cuda") if stats is None else stats
    ws = torch.full((xe.xe_correlate_packets_workspace_size(s),), 0x5A, dtype=torch.uint8, device="cuda")
    if isinstance(pk, torch.Tensor):
        pkd, n, stride = pk, pk.shape[0], pk.shape[1]
    else:
        n = pk.shape[0]
        pkd = X.dev(pk) if n else torch.empty(16, dtype=torch.uint8, device="cuda")
        stride = pk.shape[1] if n else synth.packet_stride(N)
    xe.xe_correlate_packets(pkd, n, stride, seq0, gps, s, vis, accumulate, filled, lost, stats, ws)
    return vis, filled, lost, stats


def _host(t, dtype=None):
    a = t.cpu().numpy()
    return a.astype(dtype) if dtype is not None else a


@pytest.mark.parametrize("N,F,T,gps,p_drop,p_reorder,p_dup", [
    (16, 8, 128, 1, 0.0, 0.0, 0.0),            # one tile, one group, no loss
    (64, 16, 260, 2, 0.05, 0.2, 0.05),         # ragged time tail (T % 128 = 4)
    (80, 24, 512, 3, 0.1, 0.1, 0.1),           # ragged input block (N % 64 = 16), three groups
    (192, 16, 1028, 1, 0.5, 0.5, 0.3),         # half-empty second super-block, heavy loss
    (256, 64, 256, 2, 0.02, 0.1, 0.02),        # per-server Pathfinder inputs
    (512, 8, 256, 1, 0.02, 0.1, 0.02),         # four super-blocks: doubles, off-diagonal singles, twins
    (640, 16, 132, 2, 0.05, 0.1, 0.05),        # five, the last half empty; ragged time tail
    # integrations of >= 16384 samples take the twin layout (two channels' last diagonal blocks)
    (256, 8, 16388, 1, 0.01, 0.05, 0.01),      # two doubles and a twin per channel pair; ragged tail
    (384, 8, 16384, 1, 0.01, 0.05, 0.01),      # three super-blocks: doubles, a single, a twin
])
def test_packets_match_oracle(N, F, T, gps, p_drop, p_reorder, p_dup):
    fr = synth.signal_frame(N, F, T + 64, 40 + N + T)
    seq0 = 1000
    pk = synth.packet_stream(fr, seq0 - 4, gps, seed=41 + N, p_drop=p_drop, p_reorder=p_reorder, p_dup=p_dup)
    frame_o, filled_o, lost_o, stats_o = oracle.assemble(pk, seq0, gps, N, F, T)
    vis_o, st = oracle.correlate(frame_o)
    assert st == oracle.OK
    vis, filled, lost, stats = _packets_gpu(pk, seq0, gps, N, F, T)
    np.testing.assert_array_equal(_host(vis, np.int64), vis_o)
    np.testing.assert_array_equal(_host(filled), filled_o)
    np.testing.assert_array_equal(_host(lost, np.uint32), lost_o)
    np.testing.assert_array_equal(_host(stats, np.uint32), stats_o)
    assert stats_o[2] > 0 and stats_o[3] > 0                # late and early packets were present


def test_random_packet_sets_with_64_bit_sequence_numbers():
    """Random packet sets whose sequence numbers lie far beyond 2^32 (the header's seq is a u64):
    valid, late, early, foreign-stream and foreign-group packets, and duplicates carrying different
    payloads, in random arrival order. xe_assemble and xe_correlate_packets both match the oracle's
    assembly (and its correlation of that frame) bit for bit."""
    rng = np.random.default_rng(27)
    for case in range(12):
        N = int(rng.choice([16, 32, 64]))
        gps, S, Q = int(rng.integers(1, 3)), int(rng.integers(1, 4)), int(rng.integers(1, 40))
        F, T = 8 * S * gps, 4 * Q
        seq0 = int(rng.integers(1 << 33, 1 << 50))
        n = int(rng.integers(1, 3 * Q * S * gps + 1))
        pk = synth.random_packet_set(270 + case, N, S, gps, Q, n, seq0)
        frame_o, filled_o, lost_o, stats_o = oracle.assemble(pk, seq0, gps, N, F, T)
        vis_o, st = oracle.correlate(frame_o)
        assert st == oracle.OK
        s = xe.Shape(N, F, T)
        frame = torch.full((T, F, N), 0xA5, dtype=torch.uint8, device="cuda")
        filled = torch.full((Q, F // 8), 7, dtype=torch.uint8, device="cuda")
        lost = torch.zeros(F, dtype=torch.int32, device="cuda")
        stats = torch.zeros(5, dtype=torch.int32, device="cuda")
        ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
        xe.xe_assemble(X.dev(pk), n, pk.shape[1], seq0, gps, s, frame, filled, lost, stats, ws)
        np.testing.assert_array_equal(_host(frame), frame_o, err_msg=f"case {case}: frame")
        for name, got, want in (("filled", filled, filled_o), ("lost", lost, lost_o), ("stats", stats, stats_o)):
            np.testing.assert_array_equal(_host(got, np.uint32), np.asarray(want, np.uint32), err_msg=f"case {case}: {name}")
        vis, filled2, lost2, stats2 = _packets_gpu(pk, seq0, gps, N, F, T)
        np.testing.assert_array_equal(_host(vis, np.int64), vis_o, err_msg=f"case {case}: zero-copy vis")
        assert torch.equal(filled2, filled) and torch.equal(lost2, lost) and torch.equal(stats2, stats)

def test_packets_accumulate_over_two_frames():
    """Two consecutive frames of one stream integrate into one visibility set; lost and stats
    accumulate like xe_assemble's."""
    N, F, T, gps = 64, 16, 512, 1
    fr = synth.signal_frame(N, F, 2 * T, 50)
    pk = synth.packet_stream(fr, 0, gps, seed=51, p_drop=0.05, p_reorder=0.1, p_dup=0.02)
    vis = torch.zeros((F, xe.npairs(N), 2), dtype=torch.int32, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    want = np.zeros((F, xe.npairs(N), 2), np.int64)
    lost_o = np.zeros(F, np.uint32)
    stats_o = np.zeros(5, np.uint32)
    for k in range(2):
        seq0 = k * (T // 4)
        frame_o, _, lo, so = oracle.assemble(pk, seq0, gps, N, F, T)
        v, _ = oracle.correlate(frame_o)
        want += v
        lost_o += lo
        stats_o += so
        _packets_gpu(pk, seq0, gps, N, F, T, vis=vis, accumulate=True, lost=lost, stats=stats)
    np.testing.assert_array_equal(_host(vis, np.int64), want)
    np.testing.assert_array_equal(_host(lost, np.uint32), lost_o)
    np.testing.assert_array_equal(_host(stats, np.uint32), stats_o)


def test_packets_empty_set_integrates_zero():
    N, F, T = 32, 8, 64
    pk = np.zeros((0, synth.packet_stride(N)), np.uint8)
    vis, filled, lost, stats = _packets_gpu(pk, 0, 1, N, F, T)
    assert not _host(vis).any() and not _host(filled).any()
    assert (_host(lost) == T).all() and not _host(stats).any()


def test_packets_reject_bad_geometry():
    N, F, T = 32, 8, 64
    s = xe.Shape(N, F + 4, T)                               # not whole 8-channel groups
    assert xe.xe_correlate_packets_workspace_size(s) == 0
    s = xe.Shape(N, F, T)
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    vis = torch.zeros((F, xe.npairs(N), 2), dtype=torch.int32, device="cuda")
    c = torch.zeros(16, dtype=torch.int32, device="cuda")
    pk = torch.zeros((4, synth.packet_stride(N)), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XeError) as e:                    # stride below header + payload
        xe.xe_correlate_packets(pk, 4, 16 + 16 * N, 0, 1, s, vis, False, c, c, c, ws)
    assert e.value.status == xe.XE_EINVAL
    with pytest.raises(xe.XeError) as e:                    # workspace too small
        xe.xe_correlate_packets(pk, 4, synth.packet_stride(N), 0, 1, s, vis, False, c, c, c, ws[:64])
    assert e.value.status == xe.XE_ENOMEM


def test_packets_full_band_frame_matches_two_step_path_and_oracle_sample():
    """Full-band frame (N=256, F=1024, T=4096 from 128 streams of 8 channels, 0.1% drops, in the
    launch configuration the bench times): all of vis, filled, lost and stats equal xe_assemble
    followed by xe_correlate on the device, and the oracle (assembling the same packets on the host)
    checks four channels."""
    N, F, T, gps = 256, 1024, 4096, 1
    fr = synth.signal_frame_torch(N, F, T, 60, device="cuda")
    pk = synth.packetize_torch(fr, 0, gps)
    del fr
    g = torch.Generator(device="cuda")
    g.manual_seed(61)
    keep = torch.rand(pk.shape[0], generator=g, device="cuda") >= 0.001
    pk = pk[keep].contiguous()
    s = xe.Shape(N, F, T)
    vis, filled, lost, stats = _packets_gpu(pk, 0, gps, N, F, T)
    frame = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
    filled2 = torch.empty_like(filled)
    lost2 = torch.zeros_like(lost)
    stats2 = torch.zeros_like(stats)
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_assemble(pk, pk.shape[0], pk.shape[1], 0, gps, s, frame, filled2, lost2, stats2, ws)
    vis2 = X.correlate(frame)
    del frame
    assert torch.equal(vis, vis2)
    assert torch.equal(filled, filled2) and torch.equal(lost, lost2) and torch.equal(stats, stats2)
    assert int(stats[0]) == int(keep.sum()) and int(lost.sum()) > 0
    host_pk = pk.cpu().numpy()
    del pk
    frame_o, _, lost_o, _ = oracle.assemble(host_pk, 0, gps, N, F, T)
    np.testing.assert_array_equal(_host(lost, np.uint32), lost_o)
    for f in (0, 333, 512, 1023):
        want, st = oracle.correlate(frame_o, f, 1)
        assert st == oracle.OK
        np.testing.assert_array_equal(_host(vis[f:f + 1], np.int64), want)


def test_packets_bench_launch_eight_frames_accumulating():
    """The bench's main launch at full size: the full band (N=256, F=1024, 128 streams of one
    8-channel group each) over 8 consecutive frames of T=4096 in one call (T=32768, so channel pairs
    take the twin layout), 0.1% of packets dropped, adding onto visibilities that already hold an
    earlier integration. Every channel is compared with xe_assemble followed by xe_correlate on the
    device (accumulating onto the same start values); the oracle checks two 8-channel groups, each
    assembled on the host from that group's packets alone (placement is per group, so the subset
    assembles to the same group frame)."""
    N, F, T, gps = 256, 1024, 8 * 4096, 1
    s = xe.Shape(N, F, T)
    fr = synth.signal_frame_torch(N, F, T, 70, device="cuda")
    pk = synth.packetize_torch(fr, 0, gps)
    del fr
    g = torch.Generator(device="cuda")
    g.manual_seed(71)
    keep = torch.rand(pk.shape[0], generator=g, device="cuda") >= 0.001
    pk = pk[keep].contiguous()
    torch.cuda.empty_cache()
    start = torch.randint(-(1 << 20), 1 << 20, (F, xe.npairs(N), 2), generator=g, device="cuda", dtype=torch.int32)
    vis, filled, lost, stats = _packets_gpu(pk, 0, gps, N, F, T, vis=start.clone(), accumulate=True)

    frame = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
    filled2 = torch.empty_like(filled)
    lost2 = torch.zeros_like(lost)
    stats2 = torch.zeros_like(stats)
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_assemble(pk, pk.shape[0], pk.shape[1], 0, gps, s, frame, filled2, lost2, stats2, ws)
    vis2 = X.correlate(frame, vis=start.clone(), accumulate=True)
    del frame, ws
    assert torch.equal(vis, vis2)
    assert torch.equal(filled, filled2) and torch.equal(lost, lost2) and torch.equal(stats, stats2)
    assert int(stats[0]) == int(keep.sum()) and int(lost.sum()) > 0

    sid = pk[:, :4].contiguous().view(torch.int32)[:, 0] & 0xFFFF
    for grp, chans in ((5, (0, 7)), (127, (3,))):
        sub = pk[sid == grp].clone()
        sub[:, 0:2] = 0                                     # stream id -> 0: the group alone, F = 8
        frame_o, _, lost_o, _ = oracle.assemble(sub.cpu().numpy(), 0, gps, N, 8, T)
        np.testing.assert_array_equal(_host(lost[8 * grp:8 * grp + 8], np.uint32), lost_o)
        for c in chans:
            want, st = oracle.correlate(frame_o, c, 1)
            assert st == oracle.OK
            f = 8 * grp + c
            want = want + _host(start[f:f + 1], np.int64)
            np.testing.assert_array_equal(_host(vis[f:f + 1], np.int64), want)
