"""Uneven batch in one launch (24 jobs, N 64..2048, F 16..256, T 1024..32768, signal model) on the
default CTA-pair engine, with the launch shape of every (N, T-bucket) picked by the autotuner and
installed in libxe's tuning table. Each job is checked against the oracle: whole channels where that
is cheap on the CPU, sampled visibilities otherwise; and every channel of every job equals a separate
single-job launch (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from paper_1503_06189_b300 import autotune

pytestmark = pytest.mark.gpu


def test_uneven_batch_autotuned(tmp_path, monkeypatch):
    dev = torch.device("cuda")
    shapes = synth.config4_shapes()
    monkeypatch.setattr(autotune, "PROBE_BYTES", 256 << 20)       # small probes: the test times the table, too
    table = autotune.Table(str(tmp_path / "autotune.json"))
    for N, F, T in shapes:
        table.tune_frames(N, T)
    table.install()
    try:
        installed = xe.xe_tune_table_get()
        assert len(installed) == len({(N, autotune.bucket(T)) for N, F, T in shapes})
        frames, vis, jobs = [], [], []
        for k, (N, F, T) in enumerate(shapes):
            chunk = max(1, (1 << 27) // (T * N))
            fr = synth.signal_frame_torch(N, F, T, 4000 + k, device=dev, chunk=chunk)
            v = torch.full((F, xe.npairs(N), 2), -1, dtype=torch.int32, device=dev)
            frames.append(fr)
            vis.append(v)
            jobs.append((fr, v, xe.Shape(N, F, T), False))
        ws = torch.empty(xe.xe_correlate_batched_workspace_size(jobs), dtype=torch.uint8, device=dev)
        xe.xe_correlate_batched(jobs, ws)                          # default engine, tuned launch shape
        torch.cuda.synchronize()
        _check_jobs(shapes, frames, vis, dev)
    finally:
        xe.xe_tune_table_set([])


def _check_jobs(shapes, frames, vis, dev):
    rng = np.random.default_rng(44)
    for k, ((N, F, T), fr, v) in enumerate(zip(shapes, frames, vis)):
        # every channel: equal to the job launched alone on the default (CTA-pair) engine
        alone = torch.full_like(v, -2)
        ws1 = torch.empty(xe.xe_correlate_workspace_size(xe.Shape(N, F, T)), dtype=torch.uint8, device=dev)
        xe.xe_correlate(fr, xe.Shape(N, F, T), alone, False, ws1)
        assert torch.equal(alone, v), f"job {k}: batched launch differs from a single-job launch"
        chans = sorted({0, F - 1, int(rng.integers(0, F))})
        host = fr[:, chans, :].cpu().numpy()
        got = v[chans].cpu().numpy().astype(np.int64)
        if xe.npairs(N) * T <= 3e8:                                  # whole channels
            want, st = oracle.correlate(host)
            assert st == oracle.OK
            np.testing.assert_array_equal(got, want, err_msg=f"job {k} {(N, F, T)}")
        else:                                                        # sampled visibilities
            i = rng.integers(0, N, 48)
            j = rng.integers(0, N, 48)
            pairs = np.stack([np.minimum(i, j), np.maximum(i, j)], 1)
            pairs = np.concatenate([pairs, [[0, 0], [0, N - 1], [N - 1, N - 1], [N // 2, N // 2 + 1]]])
            for c in range(len(chans)):
                want = oracle.correlate_pairs(host, c, pairs)
                idx = [oracle.pidx(int(a), int(b), N) for a, b in pairs]
                np.testing.assert_array_equal(got[c, idx], want, err_msg=f"job {k} {(N, F, T)} chan {chans[c]}")
        del fr
