"""Multi-rank host logic on CPU (gloo, world size 2): sharded trajectory
ranges reproduce a single run, and the merged tail statistics equal the
single-run statistics."""
import math
import os
import socket

import numpy as np
import pytest

import workloads as W
from paper_2410_13683_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _tail(nsteps, logw, status, dN, N_tail):
    from oracle import estimators as E
    e, p, k = E.tail_ess(nsteps, logw, status, dN, N_tail)
    return dict(p_tail=p, n_total=len(nsteps), ess_tail=e)


def _rank_main(rank, world, port, n, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import stepper as S
    from oracle import tables as T
    m = W.BM.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    off = shard.shard_offset(n, rank)
    tr = S.run(m, res, tab, seed=31, run_id=0, n=n, traj0=off, A=0.7, threads=1)
    sw, sw2 = shard.tail_sums(_tail(tr.nsteps, tr.logw, tr.status, m.dN, 5.5))
    sw, sw2 = shard.merge_tail_sums(sw, sw2, dist)
    if rank == 0:
        np.save(out_path, np.array([sw, sw2]))
    np.save(out_path + f".rank{rank}.npy", tr.nsteps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_merge_to_the_single_run(tmp_path):
    import torch.multiprocessing as mp
    n, world = 2048, 2
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), n, out), nprocs=world, join=True,
                       start_method="spawn")
    sw, sw2 = np.load(out)
    from oracle import stepper as S
    from oracle import tables as T
    m = W.BM.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    full = S.run(m, res, tab, seed=31, run_id=0, n=world * n, A=0.7, threads=2)
    for r in range(world):
        part = np.load(out + f".rank{r}.npy")
        assert np.array_equal(part, full.nsteps[r * n:(r + 1) * n])
    ref_sw, ref_sw2 = shard.tail_sums(_tail(full.nsteps, full.logw, full.status, m.dN, 5.5))
    assert sw == pytest.approx(ref_sw, rel=1e-12)
    assert sw2 == pytest.approx(ref_sw2, rel=1e-12)
    assert shard.ess_of(sw, sw2) == pytest.approx(shard.ess_of(ref_sw, ref_sw2), rel=1e-12)


def test_shard_offsets_are_disjoint_and_bounded():
    assert [shard.shard_offset(100, r) for r in range(4)] == [0, 100, 200, 300]
    with pytest.raises(ValueError):
        shard.shard_offset(1 << 31, 2)
    assert shard.merge_tail_sums(1.0, 2.0) == (1.0, 2.0)
