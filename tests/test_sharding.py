"""Multi-rank host logic on CPU (gloo, world size 2): sharded trajectory
ranges reproduce a single run, the merged tail statistics equal the
single-run statistics, and a missing shard -- a gap in the ranks' ranges, or
a rank that never reaches the merge -- is an error on every rank that
reaches it."""
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
    sw, sw2 = shard.merge_shards(sw, sw2, off, n, world * n, dist)
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
    assert shard.merge_shards(1.0, 2.0, 0, 100, 100) == (1.0, 2.0)


def test_tiling_check_names_gaps_overlaps_and_empty_shards():
    shard.check_tiling([(0, 10), (10, 5)], 15)
    shard.check_tiling([(10, 5), (0, 10)], 15)          # any rank order
    for parts, n, word in [([(0, 10), (11, 4)], 15, "missing"), ([(0, 10), (9, 6)], 15, "overlapping"),
                           ([(0, 10), (10, 0)], 10, "missing"), ([(0, 10)], 15, "missing"),
                           ([(0, 10), (10, 10)], 15, "beyond"), ([(5, 10)], 15, "missing")]:
        with pytest.raises(shard.ShardError, match=word):
            shard.check_tiling(parts, n)
    with pytest.raises(shard.ShardError, match="missing"):
        shard.merge_shards(1.0, 1.0, 0, 50, 100)          # one process that ran half the range


def _merge_main(rank, world, port, mode, out_path):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    n = 1000
    first = rank * n
    if mode == "gap" and rank == 1:
        first += 7                                       # rank 1 ran the wrong range: [1007, 2007)
    if mode == "leave" and rank == 1:
        os._exit(0)                                      # rank 1 never reaches the merge
    try:
        shard.merge_shards(1.0 + rank, 2.0, first, n, world * n, dist)
        msg = "ok"
    except shard.ShardError as e:
        msg = "ShardError: " + str(e)
    with open(out_path + f".rank{rank}", "w") as f:
        f.write(msg)
    if mode != "leave":
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["gap", "leave"])
def test_missing_shard_is_an_error_on_every_rank_that_merges(tmp_path, mode):
    import torch.multiprocessing as mp
    out = str(tmp_path / "merge")
    mp.start_processes(_merge_main, args=(2, _free_port(), mode, out), nprocs=2, join=True,
                       start_method="spawn")
    ranks = [0, 1] if mode == "gap" else [0]
    for r in ranks:
        msg = open(out + f".rank{r}").read()
        assert msg.startswith("ShardError"), (r, msg)
        if mode == "gap":
            assert "[1000, 1007)" in msg
        else:
            assert "did not take part" in msg
