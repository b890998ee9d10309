"""Block-size autotuner for the multi-shift solves.

For a call shape (m, n, mode) it times every supported n_b on seeded synthetic
inputs of that shape (workload 1's distributions for plain/conj solves,
workload 2's for the safe solve), through the same C ABI calls the user makes,
and caches the fastest per (m bucket, n bucket, mode, device name) in a JSON
file (``$MSTS_AUTOTUNE_CACHE`` or ``~/.cache/msts_autotune.json``).  The GEMM
tile and the lanes-per-shift of the diagonal step are chosen inside the library
from the launch shape; n_b is the knob left to tune.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import colmajor, msts_solve
from . import workloads as W

NB_CHOICES = (16, 32, 64)
_lock = threading.Lock()


def _cache_path() -> str:
    return os.environ.get("MSTS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "msts_autotune.json"))


def _bucket(x: int) -> int:
    b = 1
    while b < x:
        b *= 2
    return b


def _key(m, n, mode, device):
    return f"{torch.cuda.get_device_name(device)}|{mode}|m{_bucket(m)}|n{_bucket(n)}"


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


def time_nb(m, n, nb, mode="plain", device="cuda", reps=3):
    """Median milliseconds of one solve of shape (m, n) with block size nb."""
    dev = torch.device(device)
    m_t, n_t = _bucket(m), _bucket(n)
    if mode == "safe":
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
    kw = dict(safe=(mode == "safe"), conj_trans=(mode == "conj"), nb=nb)
    msts_solve(U, s, X, **kw)                      # warm-up
    times = []
    for _ in range(reps):
        X.copy_(B0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        msts_solve(U, s, X, **kw)
        e1.record()
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    return sorted(times)[len(times) // 2]


def best_nb(m, n, mode="plain", device="cuda", refresh=False):
    """The fastest n_b for this shape (cached); mode in {"plain", "safe", "conj"}."""
    key = _key(m, n, mode, device)
    with _lock:
        cache = _load()
        if not refresh and key in cache:
            return int(cache[key]["nb"])
        results = {nb: time_nb(m, n, nb, mode, device) for nb in NB_CHOICES}
        nb = min(results, key=results.get)
        cache[key] = {"nb": nb, "ms": {str(k): v for k, v in results.items()}}
        _store(cache)
        return nb
