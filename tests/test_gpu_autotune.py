"""GPU: the autotuner times every block size and caches a valid choice."""
import pytest

from paper_1607_01477_gb300 import autotune

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("MSTS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    nb = autotune.best_nb(300, 40, "plain")
    assert nb in autotune.NB_CHOICES
    cache = autotune._load()
    (key, rec), = cache.items()
    assert rec["nb"] == nb and set(rec["ms"]) == {"16", "32", "64"}
    assert autotune.best_nb(300, 40, "plain") == nb          # served from the cache
    assert autotune.best_nb(256, 64, "safe") in autotune.NB_CHOICES
