"""The multi-rank host logic of bench.py (max-over-ranks timing, summed work)
with two gloo ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.dist_init(world, "gloo")
    ms = bench.max_over_ranks(10.0 + rank, d, "cpu")
    fl = bench.sum_over_ranks(1.5, d, "cpu")
    r, w, _ = bench.dist_env()
    q.put((rank, ms, fl, r, w))
    dist.destroy_process_group()


def test_bench_reductions_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, fl, r, w in out:
        assert ms == 11.0 and fl == 3.0 and r == rank and w == 2


def test_bench_trevc_parity_flags_a_planted_error():
    """bench.py pairs its headline with the oracle on the cpu_baseline's
    columns: a correct Z passes, a perturbed column or exponent fails."""
    import numpy as np
    import torch

    import bench
    import oracle
    from paper_1607_01477_gb300 import workloads as W

    T = W.trevc_problem(96, seed=5)
    Zf, ef, _ = oracle.trevc(T, 32)
    cols = np.arange(0, 96, 2)
    Zo, eo = oracle.trevc_columns(T, cols, 32)
    Z, se = torch.from_numpy(np.asfortranarray(Zf)), torch.from_numpy(ef.astype(np.int32))
    assert bench.trevc_parity(Z, se, cols, Zo, eo)["pass"]
    Zbad = Z.clone()
    Zbad[3, 40] += 1e-6 * Zbad[:, 40].abs().max()
    assert not bench.trevc_parity(Zbad, se, cols, Zo, eo)["pass"]
    sebad = se.clone()
    sebad[10] += 1
    assert not bench.trevc_parity(Z, sebad, cols, Zo, eo)["pass"]
