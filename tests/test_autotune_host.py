"""Host-side logic of the autotuner (no GPU): buckets, keys and the cache file."""
import json

from paper_1607_01477_gb300 import autotune


def test_bucket_and_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("MSTS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    assert autotune._bucket(1) == 1 and autotune._bucket(300) == 512 and autotune._bucket(4096) == 4096
    autotune._store({"k": {"nb": 32}})
    assert autotune._load() == {"k": {"nb": 32}}
    assert json.load(open(tmp_path / "c.json"))["k"]["nb"] == 32


def test_candidates_cover_every_block_size_and_layout():
    c = autotune.candidates()
    assert {nb for nb, _ in c} == set(autotune.NB_CHOICES)
    assert {lay for nb, lay in c if nb == 32} == set(autotune.LAYOUTS)
    assert all(lay == 0 for nb, lay in c if nb != 32)
    assert len(set(c)) == len(c)
