"""F-engine flags (Sec. II-C) through the C ABI (GPU): per-input flag counts and pair intersections
from the packets' footers against the oracle, and the flagged normalisation end to end.

Flag counting is integer work: bit-exact. The end-to-end case also checks that the counter scheme
fed by the device's loss and flag counters gives the brute-force count of samples valid for both
inputs, and that the normalised matrix holds the 1e-6 relative tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu


def _flags_gpu(pk, seq0, gps, N, F, T, fc=None, fp=None):
    s = xe.Shape(N, F, T)
    fc = torch.zeros((F, N), dtype=torch.int32, device="cuda") if fc is None else fc
    fp = torch.zeros((F, xe.npairs(N)), dtype=torch.int32, device="cuda") if fp is None else fp
    ws = torch.full((xe.xe_flag_counts_workspace_size(s),), 0x5A, dtype=torch.uint8, device="cuda")
    n = pk.shape[0]
    pkd = X.dev(pk) if n else torch.empty(16, dtype=torch.uint8, device="cuda")
    stride = pk.shape[1] if n else 16 + 36 * N
    xe.xe_flag_counts(pkd, n, stride, seq0, gps, s, fc, fp, ws)
    return fc, fp


@pytest.mark.parametrize("N,F,T,gps,p_sample,p_burst,p_all", [
    (16, 8, 64, 1, 0.05, 0.1, 0.02),            # small, flags everywhere
    (64, 16, 260, 2, 0.002, 0.02, 0.002),       # sparse flags, ragged time
    (256, 16, 128, 1, 0.001, 0.01, 0.01),       # Pathfinder inputs, some fully flagged samples
])
def test_flag_counts_match_oracle(N, F, T, gps, p_sample, p_burst, p_all):
    fr = synth.signal_frame(N, F, T + 32, 70 + N)
    fl = synth.random_flags(T + 32, F, N, 71 + N, p_sample, p_burst, p_all)
    seq0 = 300
    pk = synth.packet_stream(fr, seq0 - 4, gps, seed=72 + N, p_drop=0.05, p_reorder=0.1, p_dup=0.05, flags=fl)
    want_c, want_p = oracle.flag_counts(pk, seq0, gps, N, F, T)
    fc, fp = _flags_gpu(pk, seq0, gps, N, F, T)
    np.testing.assert_array_equal(fc.cpu().numpy().astype(np.uint32), want_c)
    np.testing.assert_array_equal(fp.cpu().numpy().astype(np.uint32), want_p)
    assert want_c.sum() > 0


def test_flag_counts_accumulate_and_dense_sample():
    """Two frames accumulate; a sample with every input of a channel flagged adds one to every
    pair of that channel (the dense case)."""
    N, F, T = 32, 8, 16
    fr = synth.uniform_frame(N, F, 2 * T, 80)
    fl = np.zeros((2 * T, F, N), bool)
    fl[3, 5, :] = True                                               # frame 0: all inputs of channel 5
    fl[T + 7, 2, [1, 4, 30]] = True                                  # frame 1: three inputs of channel 2
    pk = synth.packetize(fr, 0, 1, fl)
    fc = torch.zeros((F, N), dtype=torch.int32, device="cuda")
    fp = torch.zeros((F, xe.npairs(N)), dtype=torch.int32, device="cuda")
    for k in range(2):
        _flags_gpu(pk, k * T // 4, 1, N, F, T, fc, fp)
    c = fc.cpu().numpy()
    x = fp.cpu().numpy()
    assert (c[5] == 1).all() and (x[5] == 1).all()
    assert c[2, [1, 4, 30]].tolist() == [1, 1, 1] and x[2].sum() == 6 and c.sum() == N + 3


def test_flags_end_to_end_normalisation():
    """Zero-copy correlation + flag counts + normalisation on a flagged, lossy frame: the device
    counters give the brute-force valid-sample counts, and the output holds the tolerance."""
    N, F, T, gps = 64, 16, 512, 2
    fr = synth.signal_frame(N, F, T, 90)
    fl = synth.random_flags(T, F, N, 91, p_sample=0.01, p_burst=0.05, p_all=0.005)
    pk = synth.packet_stream(fr, 0, gps, seed=92, p_drop=0.03, p_reorder=0.1, p_dup=0.02, flags=fl)
    s = xe.Shape(N, F, T)
    P = xe.npairs(N)
    pkd = X.dev(pk)
    vis = torch.empty((F, P, 2), dtype=torch.int32, device="cuda")
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_packets(pkd, pk.shape[0], pk.shape[1], 0, gps, s, vis, False, filled, lost, stats, ws)
    fc, fp = _flags_gpu(pk, 0, gps, N, F, T)
    out = torch.empty((F, P, 2), dtype=torch.float32, device="cuda")
    n_out = torch.empty((F, P), dtype=torch.int32, device="cuda")
    xe.xe_normalize(vis, s, T, lost, out, n_out, flag_count=fc, flag_pairs=fp)
    frame_o, filled_o, lost_o, _ = oracle.assemble(pk, 0, gps, N, F, T)
    vis_o, _ = oracle.correlate(frame_o)
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), vis_o)
    present = np.repeat(np.repeat(filled_o.astype(bool), 4, axis=0), 8, axis=1)
    n_mask = oracle.counts_from_mask((present[:, :, None] & ~fl).astype(np.uint8))
    np.testing.assert_array_equal(n_out.cpu().numpy().astype(np.uint32), n_mask)
    ref = oracle.normalize(vis_o, n_mask)
    o = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(o - ref) <= 1e-6 * np.abs(ref))


def test_flag_counts_reject_records_without_footer():
    N, F, T = 16, 8, 16
    s = xe.Shape(N, F, T)
    ws = torch.empty(xe.xe_flag_counts_workspace_size(s), dtype=torch.uint8, device="cuda")
    c = torch.zeros(F * xe.npairs(N), dtype=torch.int32, device="cuda")
    pk = torch.zeros((2, 16 + 32 * N), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XeError) as e:
        xe.xe_flag_counts(pk, 2, 16 + 32 * N, 0, 1, s, c, c, ws)
    assert e.value.status == xe.XE_EINVAL
