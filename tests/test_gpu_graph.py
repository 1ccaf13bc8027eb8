"""The per-frame calls captured in a CUDA graph and replayed give the oracle's results (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu


def test_graph_capture_assemble_correlate_normalize():
    N, F, T, gps = 128, 16, 512, 1
    s = xe.Shape(N, F, T)
    dev = torch.device("cuda")
    frames = [synth.signal_frame(N, F, T, 500 + k) for k in range(2)]
    pk = [synth.packet_stream(fr, k * T // 4, gps, seed=600 + k, p_drop=0.03, p_reorder=0.05) for k, fr in enumerate(frames)]
    n_max = max(p.shape[0] for p in pk)
    pkd = [torch.zeros((n_max, p.shape[1]), dtype=torch.uint8, device=dev) for p in pk]
    for d, p in zip(pkd, pk):
        d[:p.shape[0]] = torch.from_numpy(p).to(dev)
    frame = torch.empty((T, F, N), dtype=torch.uint8, device=dev)
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device=dev)
    lost = torch.zeros(F, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.int32, device=dev)
    vis = torch.empty((F, xe.npairs(N), 2), dtype=torch.int32, device=dev)
    out = torch.empty((F, xe.npairs(N), 2), dtype=torch.float32, device=dev)
    ws_a = torch.empty(xe.xe_assemble_workspace_size(s), dtype=torch.uint8, device=dev)
    ws_c = torch.empty(xe.xe_correlate_workspace_size(s), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream()

    def step():
        lost.zero_()
        for k in range(2):
            xe.xe_assemble(pkd[k], pk[k].shape[0], pk[k].shape[1], k * T // 4, gps, s, frame, filled, lost, stats,
                           ws_a, stream=stream)
            xe.xe_correlate(frame, s, vis, k > 0, ws_c, stream=stream)
        xe.xe_normalize(vis, xe.Shape(N, F, 2 * T), 2 * T, lost, out, stream=stream)

    with torch.cuda.stream(stream):
        step()                                       # eager warm-up (one-time set-up outside capture)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    vis.fill_(-1)
    out.fill_(-1.0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()

    want, lost_o = 0, np.zeros(F, np.uint32)
    for k in range(2):
        fo, _, lost_o, _ = oracle.assemble(pk[k], k * T // 4, gps, N, F, T, lost=lost_o)
        want = want + oracle.correlate(fo)[0]
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)
    ref = oracle.normalize(want, oracle.counts_from_counters(2 * T, lost_o, N))
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref))
