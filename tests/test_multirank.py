"""Ray partition across ranks (world_size 2, gloo on CPU): rank r traces rays
[r R, (r+1) R) of a 2R-ray estimate; the sum of the ranks' tallies (one binary64
all-reduce) equals the single-process estimate over all 2R rays, and the
benchmark's max-over-ranks timing reduction picks the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    import synth
    from oracle import kappa as okappa
    from oracle import trace as otrace
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = synth.config(0)
    K = okappa.kappa_table(case.lines, case.spec)
    begin, n, total = bench.ray_range(rank, world, 5000)
    r = otrace.trace(case.grid, case.spec, K, seed=case.seed, ray_begin=begin, n_rays=n, n_total=total,
                     threads=1)
    t = torch.from_numpy(np.concatenate([r.absorbed, [r.emitted, r.escaped]]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    ms = torch.tensor([10.0 + rank])
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((t.numpy(), float(ms.item())))
    dist.destroy_process_group()


def test_two_rank_partition_matches_single_process():
    import synth
    from oracle import kappa as okappa
    from oracle import trace as otrace
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, ms = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = synth.config(0)
    K = okappa.kappa_table(case.lines, case.spec)
    ref = otrace.trace(case.grid, case.spec, K, seed=case.seed, n_rays=10000, n_total=10000, threads=1)
    assert np.allclose(got[:-2], ref.absorbed, rtol=1e-12, atol=0)
    assert got[-2] == pytest.approx(ref.emitted, rel=1e-12)
    assert got[-1] == pytest.approx(ref.escaped, rel=1e-12)
    assert ms == 11.0
