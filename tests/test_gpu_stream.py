"""The streaming serving loop (xe_stream_*): results alone vs in the mix, oracle parity, admission
backpressure and latency statistics (GPU)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe

pytestmark = pytest.mark.gpu

N, GPS, T, FRAMES, S = 64, 2, 512, 5, 4
FS = 8 * GPS
Q = T // 4
P = xe.npairs(N)


def _cudart():
    torch.zeros(1, device="cuda")
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            L = ctypes.CDLL(name)
            L.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            return L
        except OSError:
            continue
    raise RuntimeError("no CUDA runtime")


def d2h(ptr, nbytes, dtype):
    out = np.empty(nbytes, np.uint8)
    assert _cudart().cudaMemcpy(out.ctypes.data, ptr, nbytes, 2) == 0
    return out.view(dtype)


def stream_packets(sid, seed, p_drop=0.02, p_reorder=0.05, p_dup=0.01):
    fr = synth.signal_frame(N, FS, T * FRAMES, seed)
    pk = synth.packetize(fr, 0, GPS)
    pk[:, 0:2] = np.frombuffer(np.uint16(sid).tobytes(), np.uint8)
    order = synth.network_order(pk.shape[0], seed + 1, p_drop, p_reorder, p_dup)
    return np.ascontiguousarray(pk[order])


def cfg(n_streams, slots=8, ring=3, max_batch=4, n_cuda_streams=2, batch_wait_us=0):
    return xe.StreamCfg(n_streams, GPS, N, T, synth.packet_stride(N), 256, ring, slots, max_batch,
                        n_cuda_streams, 0, batch_wait_us)


def collect(h, results, timeout_ms):
    while True:
        r = xe.xe_stream_poll(h, timeout_ms)
        if r is None:
            return
        results[(r.stream_id, r.frame)] = dict(
            vis=d2h(r.vis, FS * P * 8, np.int32), n=d2h(r.n, FS * P * 4, np.uint32),
            out=d2h(r.out, FS * P * 8, np.float32), lost=d2h(r.lost, FS * 4, np.uint32),
            stats=d2h(r.stats, 20, np.uint32), packets=r.packets, batch=r.batch)
        xe.xe_stream_release(h, r)
        timeout_ms = 0


def serve(packet_lists, stream_ids, chunk=96, **kw):
    """Submits the streams' packets interleaved in chunks; returns results keyed (stream, frame)."""
    h = xe.xe_stream_create(cfg(max(stream_ids) + 1, **kw))
    results, pos = {}, [0] * len(packet_lists)
    try:
        while any(p < len(pk) for p, pk in zip(pos, packet_lists)):
            for k, (sid, pk) in enumerate(zip(stream_ids, packet_lists)):
                if pos[k] >= len(pk):
                    continue
                n = min(chunk, len(pk) - pos[k])
                if xe.xe_stream_submit(h, sid, pk[pos[k]:pos[k] + n], n) == xe.XE_OK:
                    pos[k] += n
                else:
                    collect(h, results, 20)
            collect(h, results, 0)
        xe.xe_stream_flush(h)
        want = len(stream_ids) * FRAMES
        for _ in range(200):
            collect(h, results, 50)
            if len(results) >= want:
                break
        stats = xe.xe_stream_stats(h)
    finally:
        xe.xe_stream_destroy(h)
    return results, stats


@pytest.fixture(scope="module")
def packets():
    return [stream_packets(s, 900 + 10 * s) for s in range(S)]


def test_results_same_alone_and_in_the_mix(packets):
    mix, st = serve(packets, list(range(S)), batch_wait_us=3000)
    assert len(mix) == S * FRAMES
    assert st.frames_done == S * FRAMES and st.max_batch_seen >= 2       # frames were batched together
    for s in range(S):
        alone, _ = serve([packets[s]], [s])
        for k in range(FRAMES):
            a, m = alone[(s, k)], mix[(s, k)]
            for key in ("vis", "n", "out", "lost", "stats"):
                np.testing.assert_array_equal(a[key], m[key], err_msg=f"stream {s} frame {k} {key}")


def test_frames_match_oracle(packets):
    res, _ = serve(packets, list(range(S)))
    for s, k in ((0, 0), (1, 2), (3, 4)):
        pk = packets[s]
        seq = pk[:, 8:16].copy().view(np.uint64)[:, 0]
        mine = pk[(seq // Q) == k].copy()
        mine[:, 0:2] = 0                                   # the oracle assembles a single-stream frame
        fr, _, lost, stats = oracle.assemble(mine, k * Q, GPS, N, FS, T)
        vis, _ = oracle.correlate(fr)
        got = res[(s, k)]
        np.testing.assert_array_equal(got["vis"].reshape(FS, P, 2).astype(np.int64), vis)
        np.testing.assert_array_equal(got["lost"], lost)
        np.testing.assert_array_equal(got["stats"], stats)
        n = oracle.counts_from_counters(T, lost, N)
        np.testing.assert_array_equal(got["n"].reshape(FS, P), n)
        ref = oracle.normalize(vis, n)
        o = got["out"].reshape(FS, P, 2)
        assert np.all(np.abs(o - ref) <= 1e-6 * np.abs(ref))


def test_admission_backpressure_and_latency(packets):
    """With one slot and nothing released, submission must stall with XE_EAGAIN, and resume once
    the consumer releases results; latency percentiles are reported."""
    h = xe.xe_stream_create(cfg(1, slots=1, ring=2, max_batch=1, n_cuda_streams=1))
    try:
        pk = packets[0]
        pos, saw_again, results = 0, False, {}
        while pos < len(pk):
            n = min(64, len(pk) - pos)
            if xe.xe_stream_submit(h, 0, pk[pos:pos + n], n) == xe.XE_OK:
                pos += n
                continue
            saw_again = True
            collect(h, results, 50)
        assert saw_again
        xe.xe_stream_flush(h)
        for _ in range(100):
            collect(h, results, 50)
            if len(results) == FRAMES:
                break
        assert len(results) == FRAMES
        st = xe.xe_stream_stats(h)
        assert st.frames_released == FRAMES and st.latency_p50_us > 0 and st.latency_p99_us >= st.latency_p50_us
    finally:
        xe.xe_stream_destroy(h)
