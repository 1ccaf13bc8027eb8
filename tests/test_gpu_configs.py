"""Parity with the oracle at the geometries of the benchmark configurations (GPU, through the C ABI).

- Configuration 2, the per-server Pathfinder frame (N=256, F=64, T=16384, signal model): every
  channel against the oracle.
- Configuration 3, the full band (N=256, F=1024) integrated over 64 frames of T=4096 from packets
  (0.1 % lost) in the launch configuration the benchmark times (8 consecutive frames per
  xe_correlate_packets call, accumulating), then normalised: 16 channels (two 8-channel groups)
  against the oracle's assembly, correlation, counts and normalisation over all 64 frames.
- Configuration 5, the serving loop (xe_stream_*) at N=256 with 16 channel groups per stream and
  T=4096, packets with drops, reorders and duplicates: whole stream-frames against the oracle, and
  every frame identical whether its stream is served alone or mixed with the others.
- The full-CHIME scale N=2048 (F=64, T=16384): sampled visibilities against the oracle, and the
  zero-copy packet path identical to the frame path.
Correlation, assembly and counts are integer work (bit-exact); normalisation holds 1e-6 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def _host64(t):
    return t.cpu().numpy().astype(np.int64)


def test_config2_pathfinder_frame_every_channel():
    N, F, T = 256, 64, 16384
    fr = synth.signal_frame_torch(N, F, T, 2, device="cuda")
    vis = X.correlate(fr)
    want, st = oracle.correlate(fr.cpu().numpy())
    assert st == oracle.OK
    np.testing.assert_array_equal(_host64(vis), want)
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    xe.xe_normalize(vis, xe.Shape(N, F, T), T, lost, out)
    ref = oracle.normalize(want, oracle.counts_from_counters(T, np.zeros(F, np.uint32), N))
    assert np.all(np.abs(out.cpu().numpy() - ref) <= REL_TOL * np.abs(ref))


def test_config3_full_band_integration_sixteen_channels():
    N, F, T, FRAMES, PER_CALL = 256, 1024, 4096, 64, 8
    groups = (5, 77)
    Tc = PER_CALL * T
    s_call = xe.Shape(N, F, Tc)
    vis = torch.empty((F, xe.npairs(N), 2), dtype=torch.int32, device="cuda")
    filled = torch.empty((Tc // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s_call), dtype=torch.uint8, device="cuda")
    kept = 0
    host = {g: [] for g in groups}
    for c in range(FRAMES // PER_CALL):
        fr = synth.signal_frame_torch(N, F, Tc, 3000 + c, device="cuda", chunk=64)
        seq0 = c * Tc // 4
        pk = synth.packetize_torch(fr, seq0, 1)
        del fr
        g = torch.Generator(device="cuda")
        g.manual_seed(3100 + c)
        keep = torch.rand(pk.shape[0], generator=g, device="cuda") >= 0.001
        pk = pk[keep].contiguous()
        kept += pk.shape[0]
        xe.xe_correlate_packets(pk, pk.shape[0], pk.shape[1], seq0, 1, s_call, vis, c > 0, filled, lost, stats, ws)
        sid = pk[:, :4].contiguous().view(torch.int32)[:, 0] & 0xFFFF
        for grp in groups:
            sub = pk[sid == grp].clone()
            sub[:, 0:2] = 0                       # the group alone: stream 0 of an 8-channel frame
            host[grp].append(sub.cpu().numpy())
        del pk, sid
        torch.cuda.empty_cache()
    t_int = FRAMES * T
    s_int = xe.Shape(N, F, t_int)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    n_out = torch.empty((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    xe.xe_normalize(vis, s_int, t_int, lost, out, n_out)
    torch.cuda.synchronize()
    assert int(stats[0]) == kept and int(lost.sum()) > 0
    for grp in groups:
        pk = np.concatenate(host[grp])
        frame_o, _, lost_o, _ = oracle.assemble(pk, 0, 1, N, 8, t_int)
        want, st = oracle.correlate(frame_o)
        assert st == oracle.OK
        del frame_o
        f0 = 8 * grp
        np.testing.assert_array_equal(_host64(vis[f0:f0 + 8]), want, err_msg=f"group {grp}")
        np.testing.assert_array_equal(lost[f0:f0 + 8].cpu().numpy().astype(np.uint32), lost_o)
        n = oracle.counts_from_counters(t_int, lost_o, N)
        np.testing.assert_array_equal(n_out[f0:f0 + 8].cpu().numpy().astype(np.uint32), n)
        ref = oracle.normalize(want, n)
        o = out[f0:f0 + 8].cpu().numpy()
        assert np.all(np.abs(o - ref) <= REL_TOL * np.abs(ref)), f"group {grp}"


# ----------------------------------------------------------------------------- configuration 5

S5, N5, GPS5, T5, FRAMES5 = 3, 256, 16, 4096, 2
FS5 = 8 * GPS5
Q5 = T5 // 4
P5 = xe.npairs(N5)


def _stream_packets(sid, seed):
    fr = synth.signal_frame_torch(N5, FS5, T5 * FRAMES5, seed, device="cuda", chunk=32).cpu().numpy()
    pk = synth.packetize(fr, 0, GPS5)
    pk[:, 0:2] = np.frombuffer(np.uint16(sid).tobytes(), np.uint8)
    order = synth.network_order(pk.shape[0], seed + 1, p_drop=0.002, p_reorder=0.01, p_dup=0.002)
    return np.ascontiguousarray(pk[order])


def _serve(packet_lists, stream_ids, chunk=512):
    cfg = xe.StreamCfg(max(stream_ids) + 1, GPS5, N5, T5, synth.packet_stride(N5), 1024, 3, 8, 4, 2, 0, 2000)
    h = xe.xe_stream_create(cfg)
    results, pos = {}, [0] * len(packet_lists)

    def collect(timeout_ms):
        while True:
            r = xe.xe_stream_poll(h, timeout_ms)
            if r is None:
                return
            results[(r.stream_id, r.frame)] = dict(
                vis=X.d2h(r.vis, FS5 * P5 * 8, np.int32), n=X.d2h(r.n, FS5 * P5 * 4, np.uint32),
                out=X.d2h(r.out, FS5 * P5 * 8, np.float32), lost=X.d2h(r.lost, FS5 * 4, np.uint32),
                stats=X.d2h(r.stats, 20, np.uint32))
            xe.xe_stream_release(h, r)
            timeout_ms = 0

    try:
        while any(p < len(pk) for p, pk in zip(pos, packet_lists)):
            for k, (sid, pk) in enumerate(zip(stream_ids, packet_lists)):
                if pos[k] >= len(pk):
                    continue
                n = min(chunk, len(pk) - pos[k])
                if xe.xe_stream_submit(h, sid, pk[pos[k]:pos[k] + n], n) == xe.XE_OK:
                    pos[k] += n
                else:
                    collect(20)
            collect(0)
        while xe.xe_stream_flush(h) != xe.XE_OK:
            collect(20)
        for _ in range(400):
            collect(50)
            if len(results) >= len(stream_ids) * FRAMES5:
                break
        stats = xe.xe_stream_stats(h)
    finally:
        xe.xe_stream_destroy(h)
    return results, stats


def test_config5_serving_loop_full_geometry():
    packets = [_stream_packets(s, 5000 + 10 * s) for s in range(S5)]
    mix, st = _serve(packets, list(range(S5)))
    assert len(mix) == S5 * FRAMES5 and st.frames_done == S5 * FRAMES5
    assert st.latency_submit_p99_us >= st.latency_submit_p50_us > 0 and st.latency_p50_us > 0
    for s in range(S5):
        alone, _ = _serve([packets[s]], [s])
        for k in range(FRAMES5):
            a, m = alone[(s, k)], mix[(s, k)]
            for key in ("vis", "n", "out", "lost", "stats"):
                np.testing.assert_array_equal(a[key], m[key], err_msg=f"stream {s} frame {k} {key}")
    for s, k in ((0, 0), (2, 1)):
        pk = packets[s]
        seq = pk[:, 8:16].copy().view(np.uint64)[:, 0]
        mine = pk[(seq // Q5) == k].copy()
        mine[:, 0:2] = 0                                   # the oracle assembles a single-stream frame
        fr, _, lost, stats = oracle.assemble(mine, k * Q5, GPS5, N5, FS5, T5)
        vis, status = oracle.correlate(fr)
        assert status == oracle.OK
        got = mix[(s, k)]
        np.testing.assert_array_equal(got["vis"].reshape(FS5, P5, 2).astype(np.int64), vis)
        np.testing.assert_array_equal(got["lost"], lost)
        np.testing.assert_array_equal(got["stats"], stats)
        n = oracle.counts_from_counters(T5, lost, N5)
        np.testing.assert_array_equal(got["n"].reshape(FS5, P5), n)
        ref = oracle.normalize(vis, n)
        o = got["out"].reshape(FS5, P5, 2)
        assert np.all(np.abs(o - ref) <= REL_TOL * np.abs(ref))


# ----------------------------------------------------------------------------- full-CHIME scale

def test_full_chime_n2048_sampled_and_packet_path():
    N, F, T = 2048, 64, 16384
    fr = synth.signal_frame_torch(N, F, T, 2048, device="cuda", chunk=8)
    vis = X.correlate(fr)
    rng = np.random.default_rng(2048)
    chans = [0, 29, 63]
    host = fr[:, chans, :].cpu().numpy()
    i = rng.integers(0, N, 96)
    j = rng.integers(0, N, 96)
    pairs = np.stack([np.minimum(i, j), np.maximum(i, j)], 1)
    pairs = np.concatenate([pairs, [[0, 0], [0, N - 1], [N - 1, N - 1], [255, 256], [1023, 1024], [511, 1536]]])
    got = _host64(vis[chans])
    idx = [oracle.pidx(int(a), int(b), N) for a, b in pairs]
    for c, f in enumerate(chans):
        want = oracle.correlate_pairs(host, c, pairs)
        np.testing.assert_array_equal(got[c, idx], want, err_msg=f"channel {f}")
    pk = synth.packetize_torch(fr, 0, 2)
    del fr
    torch.cuda.empty_cache()
    s = xe.Shape(N, F, T)
    vis_p = torch.full_like(vis, -1)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_packets(pk, pk.shape[0], pk.shape[1], 0, 2, s, vis_p, False, filled, lost, stats, ws)
    torch.cuda.synchronize()
    assert torch.equal(vis_p, vis)
    assert int(lost.sum()) == 0 and int(stats[0]) == pk.shape[0]
