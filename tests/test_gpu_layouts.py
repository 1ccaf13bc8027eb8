"""Every item layout of the CTA-pair engine against the oracle (GPU), in both modes, through the
tuning table (the way the autotuner's choices reach a launch).

- Packet mode (xe_correlate_packets): fold, Gram with twins or wide singles, at input counts with
  whole and half super-blocks, with lost, reordered and duplicated packets.
- Frame mode (xe_correlate, xe_correlate_batched): the same layouts through the 128-sample kernel,
  which reads an assembled frame in 4-sample slots, and the 256-sample kernel
  (XE_LAYOUT_FRAME_BLOCKS); frames with T % 4 != 0 always take the latter.

Few CTA pairs per launch make every pair run several items of different kinds one after another
(the two TMEM halves alternate between them). Integer work: every comparison is bit-exact.
"""
import contextlib
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_1503_06189_b300 as xe
from paper_1503_06189_b300 import autotune
from tests import xe_cuda as X

pytestmark = pytest.mark.gpu

GRAM_LAYOUTS = [xe.XE_LAYOUT_GRAM, xe.XE_LAYOUT_GRAM_TWIN, xe.XE_LAYOUT_GRAM_WIDE]
ROW_LAYOUTS = [xe.XE_LAYOUT_AUTO, xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_FOLD_SPLIT] + GRAM_LAYOUTS


@contextlib.contextmanager
def tuned(entries):
    saved = xe.xe_tune_table_get()
    xe.xe_tune_table_set(entries)
    try:
        yield
    finally:
        xe.xe_tune_table_set(saved)


def entry(N, T, mode, layout, pairs=0, odd_pairs=-1, k_flush=0):
    return dict(n_inputs=N, t_bucket=autotune.bucket(T), mode=mode, layout=layout, pairs=pairs,
                odd_pairs=odd_pairs, k_flush=k_flush)


@functools.lru_cache(maxsize=None)
def _packet_case(N, F, T):
    """Packets of a signal-model frame with loss, reorders and duplicates, and the oracle's
    visibilities of their assembly (shared by the layouts of one shape)."""
    gps, seq0 = 1, 500
    fr = synth.signal_frame(N, F, T + 32, 60 + N)
    pk = synth.packet_stream(fr, seq0 - 4, gps, seed=61 + N, p_drop=0.02, p_reorder=0.1, p_dup=0.02)
    frame_o, _, _, _ = oracle.assemble(pk, seq0, gps, N, F, T)
    want, st = oracle.correlate(frame_o)
    assert st == oracle.OK
    return pk, want


@functools.lru_cache(maxsize=None)
def _frame_case(N, F, T):
    fr = synth.uniform_frame(N, F, T, 70 + N + T)
    want, st = oracle.correlate(fr)
    assert st == oracle.OK
    return fr, want


def _packets(pk, seq0, gps, N, F, T, vis=None, accumulate=False):
    s = xe.Shape(N, F, T)
    vis = torch.full((F, xe.npairs(N), 2), -12345, dtype=torch.int32, device="cuda") if vis is None else vis
    filled = torch.empty((T // 4, F // 8), dtype=torch.uint8, device="cuda")
    lost = torch.zeros(F, dtype=torch.int32, device="cuda")
    stats = torch.zeros(5, dtype=torch.int32, device="cuda")
    ws = torch.empty(xe.xe_correlate_packets_workspace_size(s), dtype=torch.uint8, device="cuda")
    xe.xe_correlate_packets(X.dev(pk), pk.shape[0], pk.shape[1], seq0, gps, s, vis, accumulate, filled, lost,
                            stats, ws)
    return vis


@pytest.mark.parametrize("layout", [xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_FOLD_SPLIT] + GRAM_LAYOUTS)
@pytest.mark.parametrize("N,F,T,pairs", [
    (144, 8, 388, 2),         # one super-block, a half one (16 inputs) after it
    (256, 16, 516, 3),        # one whole super-block per channel; ragged time tail
    (384, 8, 260, 5),         # a whole and a half super-block: fold, Gram diagonal, two singles
    (640, 8, 132, 7),         # two whole and a half super-block, the last 128 inputs half empty
])
def test_packet_layouts_match_oracle(layout, N, F, T, pairs):
    pk, want = _packet_case(N, F, T)
    for odd in (0, 1):
        with tuned([entry(N, T, xe.XE_TUNE_PACKETS, layout, pairs=pairs, odd_pairs=odd)]):
            vis = _packets(pk, 500, 1, N, F, T)
        np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want, err_msg=f"odd_pairs={odd}")


@pytest.mark.parametrize("layout", ROW_LAYOUTS + [xe.XE_LAYOUT_FRAME_BLOCKS])
@pytest.mark.parametrize("N,F,T,pairs", [
    (64, 5, 516, 2),          # one block per channel: twins pair channels, the fifth alone
    (256, 7, 1028, 3),        # an odd channel count; ragged time tail
    (272, 3, 260, 4),         # a whole super-block and a 16-input block
    (400, 6, 388, 0),         # a whole and a half super-block (144 inputs), all resident pairs
    (512, 3, 16388, 5),       # two super-blocks; beyond the twin threshold
])
def test_frame_layouts_match_oracle(layout, N, F, T, pairs):
    fr, want = _frame_case(N, F, T)
    with tuned([entry(N, T, xe.XE_TUNE_FRAMES, layout, pairs=pairs)]):
        vis = X.correlate(fr)
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("layout", [xe.XE_LAYOUT_AUTO, xe.XE_LAYOUT_GRAM_WIDE, xe.XE_LAYOUT_FRAME_BLOCKS])
def test_frame_layouts_accumulate(layout):
    """Two frames integrated by accumulate, onto visibilities that already hold a value."""
    N, F, T = 384, 4, 1024
    a, b = synth.signal_frame(N, F, T, 81), synth.signal_frame(N, F, T, 82)
    va, _ = oracle.correlate(a)
    vb, _ = oracle.correlate(b)
    start = np.random.default_rng(3).integers(-1000, 1000, va.shape)
    vis = X.dev(start.astype(np.int32))
    with tuned([entry(N, T, xe.XE_TUNE_FRAMES, layout, pairs=3)]):
        X.correlate(a, vis, accumulate=True)
        X.correlate(b, vis, accumulate=True)
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), start + va + vb)


@pytest.mark.parametrize("N,F,T,pairs", [(256, 13, 1028, 5), (144, 3, 260, 7), (256, 64, 516, 0), (192, 1, 132, 3),
                                         (256, 2, 4, 5)])
@pytest.mark.parametrize("accumulate", [False, True])
def test_balanced_split_matches_oracle(N, F, T, pairs, accumulate):
    """Fold items split evenly over the CTA pairs (pieces of consecutive channels, added in L2): the
    channel x stage range cut at arbitrary stages, more pairs than stages, and a call that does not
    accumulate writing over stale values. Frame and packet mode."""
    fr, want = _frame_case(N, F, T)
    start = np.random.default_rng(N + F).integers(-99, 99, want.shape)
    with tuned([entry(N, T, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_FOLD_SPLIT, pairs=pairs)]):
        vis = X.dev(start.astype(np.int32))
        X.correlate(fr, vis, accumulate=accumulate)
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want + (start if accumulate else 0))
    if F % 8 == 0:
        pk = synth.packetize(fr, 0, 1)
        with tuned([entry(N, T, xe.XE_TUNE_PACKETS, xe.XE_LAYOUT_FOLD_SPLIT, pairs=pairs)]):
            vis = _packets(pk, 0, 1, N, F, T, vis=X.dev(start.astype(np.int32)), accumulate=accumulate)
        np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want + (start if accumulate else 0))


@pytest.mark.parametrize("F", [64, 96])
def test_auto_splits_a_ragged_last_round(F):
    """Without a table entry, 96 channels of 256 inputs (two rounds of fold items on 74 pairs, the
    second a third full) take the balanced split, and 64 channels (configuration 2's shape, shorter:
    one round) one pair per channel; the result is the oracle's either way."""
    fr, want = _frame_case(256, F, 516)
    vis = X.correlate(fr)
    np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want)


def test_frame_time_not_whole_slots_takes_the_256_sample_kernel():
    """T % 4 != 0 cannot be read in 4-sample slots: the launch runs the 256-sample kernel whatever
    the table says, with the same results."""
    N, F = 256, 4
    for T in (1, 3, 130, 1031):
        fr = synth.uniform_frame(N, F, T, 90 + T)
        want, _ = oracle.correlate(fr)
        with tuned([entry(N, T, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_FOLD, pairs=2)]):
            vis = X.correlate(fr)
        np.testing.assert_array_equal(vis.cpu().numpy().astype(np.int64), want, err_msg=f"T={T}")


def test_batched_frames_mix_layouts_in_one_launch():
    """Jobs of one batched launch each take their own entry's layout (fold, Gram with twins, Gram
    with wide singles) in one 128-sample launch."""
    shapes = [(256, 5, 772), (64, 6, 1024), (384, 2, 516), (128, 3, 2048)]
    entries = [entry(256, 772, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_FOLD, pairs=4),
               entry(64, 1024, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_GRAM_TWIN),
               entry(384, 516, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_GRAM_WIDE),
               entry(128, 2048, xe.XE_TUNE_FRAMES, xe.XE_LAYOUT_GRAM)]
    frames = [synth.uniform_frame(N, F, T, 100 + k) for k, (N, F, T) in enumerate(shapes)]
    with tuned(entries):
        got = X.correlate_batched(frames)
    for fr, v in zip(frames, got):
        want, _ = oracle.correlate(fr)
        np.testing.assert_array_equal(v.cpu().numpy().astype(np.int64), want)

