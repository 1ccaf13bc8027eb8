"""Host logic of the autotuner (no GPU): T buckets, cache keys, work-item counts, the choice between
strip widths and the CTA-pair engine, and the JSON cache. The device measurement is replaced by a
fake that returns fixed timings and counts its calls."""
import json

import pytest

import paper_1503_06189_b300 as xe
from paper_1503_06189_b300 import autotune


@pytest.mark.parametrize("t,b", [(0, 128), (1, 128), (128, 128), (129, 256), (4096, 4096), (4097, 8192),
                                 (32768, 32768), (20000, 32768)])
def test_bucket_is_the_power_of_two_at_or_above_t(t, b):
    assert autotune.bucket(t) == b


def test_key_names_inputs_and_bucket():
    assert autotune.key(256, 4000) == "N256_T4096"
    assert autotune.key(2048, 1024) == "N2048_T1024"


@pytest.mark.parametrize("n", [16, 64, 100 * 16, 256, 512, 2048])
def test_strip_counts_special_cases(n):
    nb = -(-2 * n // 128)                                   # 128-row blocks of the 2N-row Gram matrix
    assert autotune._strips(n, 1) == nb * (nb + 1) // 2     # one tile per strip: every tile on/above the diagonal
    if nb <= 3:
        assert autotune._strips(n, 4) == nb                 # each row's tiles fit one strip
    counts = [autotune._strips(n, ms) for ms in (1, 2, 3, 4)]
    assert counts == sorted(counts, reverse=True)           # wider strips never need more work items


class FakeMeasure:
    def __init__(self, timings):
        self.timings = timings
        self.calls = []

    def __call__(self, n_inputs, n_time, *args, **kwargs):
        self.calls.append((n_inputs, autotune.bucket(n_time)))
        return dict(self.timings)


def test_table_picks_fastest_strip_and_caches(tmp_path, monkeypatch):
    fake = FakeMeasure({1: 3.0, 2: 1.5, 3: 2.0, 4: 1.7, "pair": 2.5})
    monkeypatch.setattr(autotune, "measure", fake)
    path = str(tmp_path / "sub" / "table.json")
    t = autotune.Table(path)
    assert t.best(256, 4000) == 2
    assert t.best_engine(256, 4000) == xe.XE_ENGINE_FUSED   # pair (2.5) slower than strip 2 (1.5)
    assert t.best(256, 4096) == 2                           # same bucket: no new measurement
    assert fake.calls == [(256, 4096)]
    t.best(256, 4097)                                       # next bucket
    assert fake.calls == [(256, 4096), (256, 8192)]
    saved = json.load(open(path))
    assert set(saved) == {"N256_T4096", "N256_T8192"} and saved["N256_T4096"]["max_strip"] == 2


def test_table_prefers_pair_engine_when_faster(monkeypatch):
    monkeypatch.setattr(autotune, "measure", FakeMeasure({1: 3.0, 2: 2.0, 3: 2.2, 4: 2.1, "pair": 1.2}))
    t = autotune.Table(None)                                # in memory only
    assert t.best_engine(2048, 32768) == xe.XE_ENGINE_FUSED_PAIR
    assert t.best(2048, 32768) == 2


def test_table_reloads_without_measuring(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "measure", FakeMeasure({1: 1.0, 2: 2.0, 3: 3.0, 4: 4.0, "pair": 5.0}))
    path = str(tmp_path / "table.json")
    autotune.Table(path).best(128, 1024)

    def no_measure(*a, **k):
        raise AssertionError("a cached bucket was measured again")

    monkeypatch.setattr(autotune, "measure", no_measure)
    t = autotune.Table(path)
    assert t.best(128, 1000) == 1 and t.best_engine(128, 1000) == xe.XE_ENGINE_FUSED
