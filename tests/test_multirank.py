"""Ray partition across ranks (world_size 2, gloo on CPU): rank r traces rays
[r R, (r+1) R) of a 2R-ray estimate; the library's combining step
(``shard.combine_tally``: one binary64 all-reduce of each rank's tally buffer)
gives the single-process estimate over all 2R rays, and the benchmark's
max-over-ranks timing reduction picks the slowest rank.  The rays are traced by
the oracle here (no GPU); the combining code is the one the benchmark runs."""
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
    import synth
    import paper_cs_0703028_gb300 as rt
    from paper_cs_0703028_gb300 import shard
    from oracle import kappa as okappa
    from oracle import trace as otrace
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = synth.config(0)
    K = okappa.kappa_table(case.lines, case.spec)
    begin, n, total = shard.ray_range(rank, world, 5000)
    r = otrace.trace(case.grid, case.spec, K, seed=case.seed, ray_begin=begin, n_rays=n, n_total=total,
                     threads=1)
    t = rt.Tally(case.grid.ncells, device="cpu")   # the rank's tally in the library's layout
    t.absorbed.copy_(torch.from_numpy(r.absorbed))
    t.scalars[0], t.scalars[1], t.scalars[2] = r.emitted, r.absorbed_total, r.escaped
    t.steps[0] = r.steps
    shard.combine_tally(t)
    ms = torch.tensor([10.0 + rank])
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((t.flat.numpy().copy(), int(t.steps.item()), float(ms.item())))
    dist.destroy_process_group()


def test_two_rank_partition_matches_single_process():
    import synth
    from paper_cs_0703028_gb300 import shard
    from oracle import kappa as okappa
    from oracle import trace as otrace
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, steps, ms = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = synth.config(0)
    nc = case.grid.ncells
    K = okappa.kappa_table(case.lines, case.spec)
    ref = otrace.trace(case.grid, case.spec, K, seed=case.seed, n_rays=10000, n_total=10000, threads=1)
    assert np.allclose(got[:nc], ref.absorbed, rtol=1e-12, atol=0)
    assert got[nc] == pytest.approx(ref.emitted, rel=1e-12)
    assert got[nc + 2] == pytest.approx(ref.escaped, rel=1e-12)
    assert steps == ref.steps
    assert shard.energy_residual(got[:nc], got[nc], got[nc + 2]) < 1e-12
    assert ms == 11.0


def test_ray_range_partitions_the_estimate():
    from paper_cs_0703028_gb300 import shard
    parts = [shard.ray_range(r, 4, 250) for r in range(4)]
    assert [p[0] for p in parts] == [0, 250, 500, 750]
    assert all(p[1] == 250 and p[2] == 1000 for p in parts)
    with pytest.raises(ValueError):
        shard.ray_range(4, 4, 250)
