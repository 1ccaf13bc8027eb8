"""The time-shift stage (xe_time_shift, xe_time_shift_counts) through the C ABI against the oracle
(GPU). The shifted frame and the counters are integer work: bit-exact. Delay spreads up to 256
samples per 128 inputs run the shared-memory window kernel (TMA boxes, zero fill before the frame's
start), larger ones the gather kernel; both are covered. End to end, packets are
assembled, shifted, correlated and normalised on the device and compared with the same chain on the
oracle (correlation bit-exact, normalisation within 1e-6 relative)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def _delays(rng, N, T, uniform_blocks=0, spread=None):
    """Delays in [0, T] (gather kernel), or within `spread` of a random offset per 128 inputs
    (window kernel when spread <= 256)."""
    if spread is None:
        d = rng.integers(0, T + 1, N)
        d[0], d[-1] = 0, T                                  # no shift, and nothing left
    else:
        off = rng.integers(0, max(1, T - spread) + 1, (N + 127) // 128)
        off[0] = 0                                          # the first block starts unshifted
        d = np.minimum(np.repeat(off, 128)[:N] + rng.integers(0, spread + 1, N), T)
        d[0] = 0
    for b in range(uniform_blocks):                         # some blocks of 16 inputs share one delay
        d[16 * b:16 * b + 16] = d[16 * b]
    return d


def _shift_gpu(fr, d):
    T, F, N = fr.shape
    src = X.dev(fr)
    out = torch.full_like(src, 0xA5)
    xe.xe_time_shift(src, xe.Shape(N, F, T), d, out)
    return out


@pytest.mark.parametrize("N,F,T,ub", [(16, 3, 37, 0), (48, 2, 300, 1), (64, 5, 1, 2), (256, 8, 4100, 8),
                                      (272, 2, 513, 3), (1024, 1, 200, 0)])
def test_time_shift_matches_oracle(N, F, T, ub):
    rng = np.random.default_rng(N + T)
    fr = synth.uniform_frame(N, F, T, 3 * N + T)
    d = _delays(rng, N, T, ub)
    got = _shift_gpu(fr, d).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.time_shift(fr, d))


@pytest.mark.parametrize("N,F,T,ub,spread", [(16, 3, 37, 0, 5), (48, 2, 300, 1, 40), (64, 5, 129, 2, 0),
                                             (256, 8, 4100, 8, 256), (272, 3, 513, 3, 17), (1024, 2, 1000, 20, 200),
                                             (128, 4, 700, 4, 256)])
def test_time_shift_window_kernel_matches_oracle(N, F, T, ub, spread):
    """Spreads of at most 256 samples per 128 inputs: the window kernel, with tiles cut by T and N,
    boxes narrower than 128 inputs (N < 128), and delays larger than the tile's first row."""
    rng = np.random.default_rng(N + T + spread)
    fr = synth.uniform_frame(N, F, T, 5 * N + T)
    d = _delays(rng, N, T, ub, spread)
    got = _shift_gpu(fr, d).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.time_shift(fr, d))


def test_time_shift_zero_delays_and_empty_frame():
    fr = synth.uniform_frame(32, 2, 64, 9)
    np.testing.assert_array_equal(_shift_gpu(fr, np.zeros(32, int)).cpu().numpy(), fr)
    a = torch.zeros(16, dtype=torch.uint8, device="cuda")
    b = torch.zeros(16, dtype=torch.uint8, device="cuda")
    xe.xe_time_shift(a, xe.Shape(32, 2, 0), np.zeros(32, int), b)           # T = 0: nothing to do


def test_time_shift_counts_match_oracle():
    rng = np.random.default_rng(5)
    N, F, T = 80, 3, 1000
    d = _delays(rng, N, T, 2)
    c0 = rng.integers(0, 50, (F, N)).astype(np.uint32)
    x0 = rng.integers(0, 50, (F, xe.npairs(N))).astype(np.uint32)
    c = X.dev(c0.view(np.int32))
    x = X.dev(x0.view(np.int32))
    xe.xe_time_shift_counts(d, xe.Shape(N, F, T), c, x)
    wc, wx = oracle.time_shift_counts(d, N, F, c0.copy(), x0.copy())
    np.testing.assert_array_equal(c.cpu().numpy().view(np.uint32), wc)
    np.testing.assert_array_equal(x.cpu().numpy().view(np.uint32), wx)


def test_time_shift_rejects_bad_arguments():
    N, F, T = 32, 2, 64
    s = xe.Shape(N, F, T)
    a = torch.zeros((T, F, N), dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    for bad in (np.full(N, T + 1), np.full(N, -1)):
        with pytest.raises(xe.XeError):
            xe.xe_time_shift(a, s, bad, b)
    with pytest.raises(xe.XeError):                           # in place is not supported
        xe.xe_time_shift(a, s, np.zeros(N, int), a)
    with pytest.raises(ValueError):                           # one delay per input
        xe.xe_time_shift(a, s, np.zeros(N - 1, int), b)


def test_time_shift_realigns_delayed_source():
    """A common source reaching input n tau_n samples late, re-aligned by delays D - tau_n: the
    correlation equals g_i conj(g_j) times the source power over the samples both inputs keep."""
    rng = np.random.default_rng(7)
    N, T, D = 64, 2048, 100
    tau = rng.integers(0, D + 1, N)
    tau[0] = D
    g = rng.integers(-1, 2, N) + 1j * rng.integers(-1, 2, N)
    s_t = rng.integers(-3, 4, T + D) + 1j * rng.integers(-3, 4, T + D)
    x = np.stack([g[n] * s_t[D - tau[n]:D - tau[n] + T] for n in range(N)], axis=1)
    fr = synth.pack(x.real.astype(np.int64), x.imag.astype(np.int64))[:, None, :]
    d = D - tau
    vis = X.correlate(_shift_gpu(fr, d)).cpu().numpy().astype(np.int64)
    mag2 = (s_t.real.astype(np.int64) ** 2 + s_t.imag.astype(np.int64) ** 2)[:T]   # |s(t - D)|^2 at t = 0 .. T - 1
    power = np.cumsum(mag2[::-1])[::-1]                                            # power[t0] = sum over t >= t0
    for i in range(0, N, 7):
        for j in range(i, N, 5):
            want = g[i] * np.conj(g[j]) * power[max(d[i], d[j])]
            p = oracle.pidx(i, j, N)
            assert vis[0, p, 0] == want.real and vis[0, p, 1] == want.imag, (i, j)


def test_time_shift_in_the_frame_pipeline():
    """Packets (with loss and reordering) -> xe_assemble -> xe_time_shift -> xe_correlate ->
    xe_time_shift_counts + xe_normalize, against the same chain on the oracle."""
    rng = np.random.default_rng(11)
    N, F, T, gps = 256, 16, 2048, 1
    s = xe.Shape(N, F, T)
    fr = synth.signal_frame(N, F, T, 12)
    pk = synth.packet_stream(fr, 0, gps, seed=13, p_drop=0.01, p_reorder=0.05, p_dup=0.01)
    d = _delays(rng, N, 300, 4)
    frame = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
    shifted = torch.empty_like(frame)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_assemble(X.dev(pk), pk.shape[0], pk.shape[1], 0, gps, s, frame, filled, lost, stats, ws)
    xe.xe_time_shift(frame, s, d, shifted)
    vis = X.correlate(shifted)
    c = torch.zeros((F, N), dtype=torch.int32, device="cuda")
    x = torch.zeros((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    xe.xe_time_shift_counts(d, s, c, x)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device="cuda")
    n_out = torch.empty((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    xe.xe_normalize(vis, s, T, lost, out, n_out, flag_count=c, flag_pairs=x)
    torch.cuda.synchronize()

    fo, _, lost_o, _ = oracle.assemble(pk, 0, gps, N, F, T)
    want, st = oracle.correlate(oracle.time_shift(fo, d))
    assert st == oracle.OK
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)
    co, xo = oracle.time_shift_counts(d, N, F)
    n = oracle.counts_from_counters(T, lost_o, N, co, xo)
    np.testing.assert_array_equal(n_out.cpu().numpy().view(np.uint32), n)
    ref = oracle.normalize(want, n)
    o = out.cpu().numpy()
    assert np.all(np.abs(o - ref) <= REL_TOL * np.abs(ref))


def _block_delays(rng, N, T, hi):
    """One delay per block of 16 inputs, in [0, min(hi, T)], expanded to one per input; the first
    block unshifted and, where T allows, one block shifted by the whole frame."""
    b = rng.integers(0, min(hi, T) + 1, N // 16)
    b[0] = 0
    if N >= 64:
        b[-1] = T
    return np.repeat(b, 16)


def _shifted_packets(pk, N, F, T, gps, d, accumulate=False, vis=None):
    s = xe.Shape(N, F, T)
    vis = torch.zeros((F, xe.npairs(N), 2), dtype=torch.int32, device="cuda") if vis is None else vis
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_packets_shifted(X.dev(pk), pk.shape[0], pk.shape[1], 0, gps, s, d, vis, accumulate, filled,
                                    lost, stats, ws)
    torch.cuda.synchronize()
    return vis, filled, lost, stats


@pytest.mark.parametrize("N,F,T,hi", [(256, 16, 4096, 300),    # fold items (one per channel)
                                      (512, 8, 2048, 2048),    # fold items and Gram singles between super-blocks
                                      (128, 16, 16384, 700),   # Gram blocks, twins (T >= 16384)
                                      (64, 8, 1028, 1028),     # Gram blocks, wide singles; ragged time tail
                                      (272, 8, 516, 64),       # a half super-block at the end (Gram single)
                                      (16, 8, 4, 4)])          # one slot
def test_shifted_packets_match_oracle(N, F, T, hi):
    """xe_correlate_packets_shifted (delays applied while the packets are read) equals assembly,
    time shift and correlation on the oracle, bit for bit, with lost, duplicated and reordered
    packets; the index outputs equal xe_correlate_packets'."""
    rng = np.random.default_rng(N * 7 + T)
    gps = 1
    fr = synth.uniform_frame(N, F, T, N + 5 * T)
    pk = synth.packet_stream(fr, 0, gps, seed=N + T, p_drop=0.02, p_reorder=0.05, p_dup=0.02)
    d = _block_delays(rng, N, T, hi)
    vis, filled, lost, stats = _shifted_packets(pk, N, F, T, gps, d)
    fo, filled_o, lost_o, _ = oracle.assemble(pk, 0, gps, N, F, T)
    want, st = oracle.correlate(oracle.time_shift(fo, d))
    assert st == oracle.OK
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)
    np.testing.assert_array_equal(lost.cpu().numpy().astype(np.int64), lost_o.astype(np.int64))
    np.testing.assert_array_equal(filled.cpu().numpy(), filled_o)


def test_shifted_packets_equal_the_two_pass_path_and_accumulate():
    """Full-band geometry, 8 frames per call, accumulating onto earlier visibilities: the fused path
    equals xe_assemble -> xe_time_shift -> xe_correlate on the device, and on sampled channels the
    oracle."""
    rng = np.random.default_rng(21)
    N, F, T, gps = 256, 64, 8192, 8
    s = xe.Shape(N, F, T)
    fr = synth.signal_frame(N, F, T, 22)
    pk = synth.packet_stream(fr, 0, gps, seed=23, p_drop=0.001, p_reorder=0.005, p_dup=0.001)
    d = _block_delays(rng, N, T, 4096)
    start = torch.randint(-1000, 1000, (F, xe.npairs(N), 2), dtype=torch.int32, device="cuda")
    vis, _, _, _ = _shifted_packets(pk, N, F, T, gps, d, accumulate=True, vis=start.clone())
    frame = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
    shifted = torch.empty_like(frame)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_assemble(X.dev(pk), pk.shape[0], pk.shape[1], 0, gps, s, frame, filled, lost, stats, ws)
    xe.xe_time_shift(frame, s, d, shifted)
    two = X.correlate(shifted, start.clone(), accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(vis.cpu().numpy(), two.cpu().numpy())
    fo, _, _, _ = oracle.assemble(pk, 0, gps, N, F, T)
    so = oracle.time_shift(fo, d)
    for f in (0, 17, 63):
        want, _ = oracle.correlate(np.ascontiguousarray(so[:, f:f + 1, :]))
        np.testing.assert_array_equal(vis[f].cpu().numpy().astype(np.int64) - start[f].cpu().numpy(), want[0])


def test_shifted_packets_zero_delays_equal_unshifted_and_reject_bad_delays():
    """Zero delays give xe_correlate_packets' result; delays out of [0, T] or differing within a block
    of 16 inputs are rejected before any work."""
    N, F, T, gps = 256, 8, 1024, 1
    s = xe.Shape(N, F, T)
    fr = synth.uniform_frame(N, F, T, 31)
    pk = synth.packet_stream(fr, 0, gps, seed=32, p_drop=0.01, p_reorder=0.02, p_dup=0.01)
    vis0, _, _, _ = _shifted_packets(pk, N, F, T, gps, np.zeros(N, int))
    ref = torch.zeros_like(vis0)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_packets(X.dev(pk), pk.shape[0], pk.shape[1], 0, gps, s, ref, False, filled, lost, stats, ws)
    torch.cuda.synchronize()
    assert torch.equal(vis0, ref)
    bad = [np.full(N, -1), np.full(N, T + 1), np.r_[np.zeros(N - 1, int), 1]]
    for d in bad:
        with pytest.raises(xe.XeError):
            _shifted_packets(pk, N, F, T, gps, d)


def test_shifted_packets_balanced_split():
    """The shifted reads in a launch whose pieces start part-way into a channel (XE_LAYOUT_FOLD_SPLIT,
    80 channels of 5 stages on at most 74 pairs): pieces begin kt0 stages in, at the delayed slots."""
    rng = np.random.default_rng(41)
    N, F, T, gps = 256, 80, 516, 1
    fr = synth.uniform_frame(N, F, T, 42)
    pk = synth.packet_stream(fr, 0, gps, seed=43, p_drop=0.02, p_reorder=0.05, p_dup=0.02)
    d = _block_delays(rng, N, T, 400)
    saved = xe.xe_tune_table_get()
    xe.xe_tune_table_set([dict(n_inputs=N, t_bucket=1024, mode=xe.XE_TUNE_PACKETS, layout=xe.XE_LAYOUT_FOLD_SPLIT,
                               pairs=0, odd_pairs=0, k_flush=0)])
    try:
        vis, _, _, _ = _shifted_packets(pk, N, F, T, gps, d)
    finally:
        xe.xe_tune_table_set(saved)
    fo, _, _, _ = oracle.assemble(pk, 0, gps, N, F, T)
    want, _ = oracle.correlate(oracle.time_shift(fo, d))
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)
