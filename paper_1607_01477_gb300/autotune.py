"""Autotuner for the multi-shift solves: block size n_b and the layout of the
diagonal-block step.

For a call kind -- ``plain``, ``safe`` or ``conj`` multi-shift solve, ``trevc``,
``pseudo`` (Lanczos pseudospectra) or ``batched`` -- and a shape, it times every
candidate on seeded synthetic inputs of that shape (the workloads' own
distributions), through the same C ABI calls the user makes, and caches the
fastest per (device name, kind, substitution path, m bucket, n bucket) in a JSON
file (``$MSTS_AUTOTUNE_CACHE`` or ``~/.cache/msts_autotune.json``).

Candidates: n_b in {16, 32, 64}, and for n_b = 32 the layout of the
diagonal-block step (``MSTS_TUNE_DIAG_LANES``): the library's own per-launch
choice from its measured tables (0), the one-warp layout (-1), or the four-warp
layout with 1, 2 or 4 lanes per shift.  The layouts give the same results bit
for bit; n_b changes the blocking and therefore the rounding, not the accuracy
class.  The GEMM tiles follow the launch shape inside the library.

The binding calls ``choose`` when a function is given ``nb=None`` and applies
the choice for the duration of that call (``applied``); the knob is
process-wide, so tuned calls should not be issued from several host threads
at once.
"""
from __future__ import annotations

import contextlib
import json
import math
import os
import threading

import torch

from . import workloads as W

NB_CHOICES = (16, 32, 64)
LAYOUTS = (0, -1, 1, 2, 4)
KINDS = ("plain", "safe", "conj", "trevc", "pseudo", "batched")
TUNE_DIAG_LANES = 1
_lock = threading.RLock()


def candidates():
    """(nb, layout) pairs: every n_b with the library's choice, and every layout at n_b = 32."""
    return [(nb, 0) for nb in NB_CHOICES] + [(32, lay) for lay in LAYOUTS if lay != 0]


def _cache_path() -> str:
    return os.environ.get("MSTS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "msts_autotune.json"))


def _bucket(x: int) -> int:
    b = 1
    while b < x:
        b *= 2
    return b


def _key(kind, m, n, tensor, device):
    return f"{torch.cuda.get_device_name(device)}|{kind}|{'tensor' if tensor else 'fp64'}|m{_bucket(m)}|n{_bucket(n)}"


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    path = _cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


@contextlib.contextmanager
def applied(layout):
    """Sets the diagonal-step layout knob for the duration of a call."""
    from . import load_library
    lib = load_library()
    if lib.msts_tune_set(TUNE_DIAG_LANES, int(layout)) != 0:
        raise ValueError(f"invalid diagonal-step layout {layout}")
    try:
        yield
    finally:
        lib.msts_tune_set(TUNE_DIAG_LANES, 0)


def _runner(kind, m, n, tensor, dev):
    """A closure running one call of this kind and shape with given (nb, layout)."""
    from . import (colmajor, msts_pseudospectra, msts_solve, msts_solve_batched, msts_trevc)
    m_t, n_t = _bucket(m), _bucket(n)
    if kind == "trevc":
        T = colmajor(torch.from_numpy(W.trevc_problem(m_t, seed=11)).to(dev))
        return lambda nb: msts_trevc(T, nb=nb, tensor=tensor)
    if kind == "pseudo":
        # two Lanczos steps: the per-step work of the full run, in proportion
        Tn, zn, Vn = W.pseudo_problem(m_t, grid=max(1, int(math.ceil(n_t ** 0.5))), seed=11)
        T = colmajor(torch.from_numpy(Tn).to(dev))
        z = torch.from_numpy(zn[:n_t]).to(dev)
        V = colmajor(torch.from_numpy(Vn[:, :n_t].copy()).to(dev))
        return lambda nb: msts_pseudospectra(T, z, V, 2, nb=nb, tensor=tensor)
    if kind == "batched":
        # n is the batch size; m the largest order (orders spread over [m/8, m])
        probs = W.batch_problem(batch=max(1, n), m_lo=max(1, m // 8), m_hi=max(1, m), n=32, seed=11)
        dp = [(colmajor(torch.from_numpy(U).to(dev)), torch.from_numpy(s).to(dev),
               colmajor(torch.from_numpy(B).to(dev))) for U, s, B in probs]
        Xs = [B.clone() for _, _, B in dp]

        def run(nb):
            for X, (_, _, B) in zip(Xs, dp):
                X.copy_(B)
            return msts_solve_batched([(U, s, X) for (U, s, _), X in zip(dp, Xs)], nb=nb, tensor=tensor)
        return run
    if kind == "safe":
        T = W.trevc_problem(m_t, seed=11)
        U = colmajor(torch.from_numpy(T).to(dev))
        g = W.rng(0, 12)
        s = torch.from_numpy(W.disk(g, n_t, 1.0)).to(dev)
        B0 = colmajor(torch.from_numpy(W.cn(g, (m_t, n_t))).to(dev))
    else:
        Un, sn, Bn = W.plain_problem(m_t, n_t, seed=11)
        U = colmajor(torch.from_numpy(Un).to(dev))
        s = torch.from_numpy(sn).to(dev)
        B0 = colmajor(torch.from_numpy(Bn).to(dev))
    X = B0.clone()
    return lambda nb: msts_solve(U, s, X.copy_(B0), safe=(kind == "safe"), conj_trans=(kind == "conj"),
                                 nb=nb, tensor=tensor)


def time_candidates(kind, m, n, tensor=False, device="cuda", reps=3):
    """Median milliseconds of every candidate (nb, layout) for this kind and shape."""
    if kind not in KINDS:
        raise ValueError(f"unknown kind {kind}")
    dev = torch.device(device)
    run = _runner(kind, m, n, tensor, dev)
    out = {}
    for nb, lay in candidates():
        with applied(lay):
            run(nb)                                   # warm-up (kernel attributes, caches)
            torch.cuda.synchronize(dev)
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                run(nb)
                e1.record()
                torch.cuda.synchronize(dev)
                times.append(e0.elapsed_time(e1))
        out[(nb, lay)] = sorted(times)[len(times) // 2]
    return out


def choose(kind, m, n, tensor=False, device="cuda", refresh=False):
    """The fastest (nb, layout) for this call kind and shape (cached)."""
    key = _key(kind, m, n, tensor, device)
    with _lock:
        cache = _load()
        if not refresh and key in cache:
            rec = cache[key]
            return int(rec["nb"]), int(rec["layout"])
        results = time_candidates(kind, m, n, tensor, device)
        nb, lay = min(results, key=results.get)
        cache[key] = {"nb": nb, "layout": lay, "ms": {f"{a},{b}": v for (a, b), v in results.items()}}
        _store(cache)
        return nb, lay


def best_nb(m, n, mode="plain", device="cuda", refresh=False):
    """The block size of the fastest candidate for a multi-shift solve of this shape."""
    return choose(mode, m, n, False, device, refresh)[0]
