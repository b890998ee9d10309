"""GPU: the autotuner times every candidate (n_b x diagonal-step layout) for
each call kind, caches a valid choice, and the binding applies it when given
nb=None; a tuned call's result equals the same call with the chosen n_b given
explicitly (the layout changes no bit)."""
import numpy as np
import pytest
import torch

import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import autotune
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("MSTS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    nb = autotune.best_nb(300, 40, "plain")
    assert nb in autotune.NB_CHOICES
    cache = autotune._load()
    (key, rec), = cache.items()
    assert rec["nb"] == nb and len(rec["ms"]) == len(autotune.candidates())
    assert autotune.best_nb(300, 40, "plain") == nb          # served from the cache
    assert autotune.best_nb(256, 64, "safe") in autotune.NB_CHOICES


@pytest.mark.parametrize("kind,m,n,tensor", [("trevc", 200, 200, True), ("pseudo", 120, 64, True),
                                             ("batched", 160, 4, False), ("conj", 150, 40, False)])
def test_every_kind_is_tuned(tmp_path, monkeypatch, kind, m, n, tensor):
    monkeypatch.setenv("MSTS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    nb, lay = autotune.choose(kind, m, n, tensor)
    assert nb in autotune.NB_CHOICES and lay in autotune.LAYOUTS
    assert (nb == 32) or lay == 0


def test_binding_applies_the_tuned_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("MSTS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    U, s, B = W.plain_problem(300, 40, seed=77)
    Ud, sd = to_dev(U), to_dev(s)
    Xa = to_dev(B)
    msts.msts_solve(Ud, sd, Xa, nb=None, tensor=True)             # tunes, then solves
    nb, lay = autotune.choose("plain", 300, 40, True)
    Xb = to_dev(B)
    msts.msts_solve(Ud, sd, Xb, nb=nb, tensor=True)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb)
    T = W.trevc_problem(200, seed=5)
    Z1, _, se1, _ = msts.msts_trevc(to_dev(T), nb=None)
    nb_t, _ = autotune.choose("trevc", 200, 200, False)
    Z2, _, se2, _ = msts.msts_trevc(to_dev(T), nb=nb_t)
    assert torch.equal(Z1, Z2) and torch.equal(se1, se2)
