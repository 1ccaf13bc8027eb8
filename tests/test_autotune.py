"""Host logic of the autotuner (no GPU): T buckets, cache keys, work-item counts per layout (against
the enumeration the kernel uses, written out), candidate sets, the choice of the fastest candidate,
the JSON cache, and installing the table into libxe (a host-only call). The device measurement is
replaced by a fake that returns fixed timings and counts its calls."""
import json

import pytest

import paper_1503_06189_b300 as xe
from paper_1503_06189_b300 import autotune


@pytest.mark.parametrize("t,b", [(0, 128), (1, 128), (128, 128), (129, 256), (4096, 4096), (4097, 8192),
                                 (32768, 32768), (20000, 32768)])
def test_bucket_is_the_power_of_two_at_or_above_t(t, b):
    assert autotune.bucket(t) == b


def test_key_names_mode_inputs_and_bucket():
    assert autotune.key("packets", 256, 4000) == "packets_N256_T4096"
    assert autotune.key("frames", 2048, 1024) == "frames_N2048_T1024"


def _fold_cover(nb):
    """Blocks (R, C) of a channel covered by the fold layout, item by item (fold items cover three)."""
    cover = []
    for q in range(nb // 2):
        cover += [(2 * q, 2 * q), (2 * q, 2 * q + 1), (2 * q + 1, 2 * q + 1)]
    if nb & 1:
        cover.append((nb - 1, nb - 1))
    for r in range(nb):
        for c in range(2 * (r // 2 + 1), nb):
            cover.append((r, c))
    return cover


@pytest.mark.parametrize("n", [144, 256, 272, 384, 512, 640, 2048, 4096])
def test_fold_layout_covers_every_block_once(n):
    nb = autotune.blocks(n)
    cover = _fold_cover(nb)
    assert sorted(cover) == sorted((r, c) for r in range(nb) for c in range(r, nb))
    fold_items = nb // 2
    assert autotune.items_per_channel(n, xe.XE_LAYOUT_FOLD, 4096) == len(cover) - 2 * fold_items


def test_items_per_channel_of_the_gram_layouts():
    # N = 256: one double and a twin half or a wide single per channel
    assert autotune.items_per_channel(256, xe.XE_LAYOUT_GRAM_TWIN, 4096) == 1.5
    assert autotune.items_per_channel(256, xe.XE_LAYOUT_GRAM_WIDE, 32768) == 2.0
    assert autotune.items_per_channel(256, xe.XE_LAYOUT_GRAM, 32768) == 1.5    # twins from T >= 16384
    assert autotune.items_per_channel(256, xe.XE_LAYOUT_AUTO, 4096) == 1       # fold at N > 128
    assert autotune.items_per_channel(64, xe.XE_LAYOUT_AUTO, 4096) == 1        # one block: wide single
    assert autotune.items_per_channel(2048, xe.XE_LAYOUT_FRAME_BLOCKS, 0) == 136   # 256-sample kernel


def test_candidate_sets():
    p256 = autotune.packet_candidates(256)
    assert {c["layout"] for c in p256} == {xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_GRAM, xe.XE_LAYOUT_FOLD_SPLIT}
    assert {c["layout"] for c in autotune.packet_candidates(512)} == {xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_GRAM}
    assert {c["odd_pairs"] for c in p256} == {0, 1}
    p64 = autotune.packet_candidates(64)
    assert {c["layout"] for c in p64} == {xe.XE_LAYOUT_GRAM_TWIN, xe.XE_LAYOUT_GRAM_WIDE}
    f = autotune.frame_candidates(256, 100)
    assert {c["layout"] for c in f} == {xe.XE_LAYOUT_FOLD, xe.XE_LAYOUT_GRAM, xe.XE_LAYOUT_FOLD_SPLIT,
                                        xe.XE_LAYOUT_FRAME_BLOCKS}
    blk = [c for c in f if c["layout"] == xe.XE_LAYOUT_FRAME_BLOCKS]
    assert {c["pairs"] for c in blk} == {0, 60}       # 300 blocks: 5 rounds on 74 pairs, 60 pairs suffice
    # T % 4 != 0: only the 256-sample kernel reads such a frame
    assert {c["layout"] for c in autotune.frame_candidates(256, 100, 1030)} == {xe.XE_LAYOUT_FRAME_BLOCKS}


def test_probe_channels_aim_for_rounds_within_bytes():
    assert autotune.probe_chan(256, 4096, 1, 8) == 296
    assert autotune.probe_chan(2048, 32768, 136, 1) == 2
    assert autotune.probe_chan(256, 1 << 20, 1, 8) == 8               # capped by the probe's bytes


class FakeMeasure:
    def __init__(self, timings):
        self.timings = timings
        self.calls = []

    def __call__(self, n_inputs, n_time, *args, **kwargs):
        self.calls.append((n_inputs, autotune.bucket(n_time)))
        return [(dict(c), ms) for c, ms in self.timings]


def test_table_picks_fastest_candidate_caches_and_installs(tmp_path, monkeypatch):
    fold = dict(layout=xe.XE_LAYOUT_FOLD, pairs=0, odd_pairs=0, k_flush=0)
    gram = dict(layout=xe.XE_LAYOUT_GRAM, pairs=0, odd_pairs=1, k_flush=0)
    fake = FakeMeasure([(fold, 4.6), (gram, 5.1)])
    monkeypatch.setattr(autotune, "measure_packets", fake)
    monkeypatch.setattr(autotune, "measure_frames", FakeMeasure([(dict(fold, layout=0, pairs=64), 9.0)]))
    path = str(tmp_path / "sub" / "table.json")
    t = autotune.Table(path)
    e = t.tune_packets(256, 32768)
    assert e["layout"] == xe.XE_LAYOUT_FOLD and e["ms"] == 4.6 and len(e["measured"]) == 2
    t.tune_packets(256, 20000)                                     # same bucket: no new measurement
    assert fake.calls == [(256, 32768)]
    t.tune_frames(2048, 16384)
    saved = json.load(open(path))
    assert set(saved) == {"packets_N256_T32768", "frames_N2048_T16384"}
    t2 = autotune.Table(path)                                      # reloaded from the cache
    assert t2.tune_packets(256, 32768)["layout"] == xe.XE_LAYOUT_FOLD and fake.calls == [(256, 32768)]
    try:
        t2.install()
        got = {(e["n_inputs"], e["t_bucket"], e["mode"]): e for e in xe.xe_tune_table_get()}
        assert got[(256, 32768, xe.XE_TUNE_PACKETS)]["layout"] == xe.XE_LAYOUT_FOLD
        assert got[(2048, 16384, xe.XE_TUNE_FRAMES)]["pairs"] == 64
    finally:
        xe.xe_tune_table_set([])


def test_tune_table_rejects_bad_entries():
    good = dict(n_inputs=256, t_bucket=4096, mode=0, layout=4, pairs=0, odd_pairs=-1, k_flush=0)
    for bad in (dict(good, t_bucket=4000), dict(good, n_inputs=250), dict(good, layout=9), dict(good, mode=2),
                dict(good, k_flush=100), dict(good, odd_pairs=2),
                dict(good, layout=xe.XE_LAYOUT_FRAME_BLOCKS)):           # the 256-sample kernel: frames only
        with pytest.raises(xe.XeError) as e:
            xe.xe_tune_table_set([bad])
        assert e.value.status == xe.XE_EINVAL
    for bad in (dict(good, layout=7), dict(good, layout=-1)):
        with pytest.raises(xe.XeError) as e:
            xe.xe_tune_table_set([bad])
        assert e.value.status == xe.XE_EINVAL
    with pytest.raises(xe.XeError):
        xe.xe_tune_table_set([good, dict(good)])                  # two entries for one (N, bucket, mode)
    xe.xe_tune_table_set([good, dict(good, mode=1, layout=xe.XE_LAYOUT_FRAME_BLOCKS)])
    assert len(xe.xe_tune_table_get()) == 2
    xe.xe_tune_table_set([])
    assert xe.xe_tune_table_get() == []
