"""The multi-GPU bench runs independent replicas: every rank holds its own
key and coins, no data moves between ranks, and the whole-job time is the
slowest rank's.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2606_01211_gb300.inputs import coins, master_seeds
    key_seed, coin_seed = bench.replica_seeds(rank)
    local = [1.5, 4.0][rank]
    t = bench.max_over_ranks(local, dist, torch.device("cpu"))
    ms = master_seeds(1, seed=key_seed)[0].tobytes()
    cs = coins(4, seed=coin_seed)[0].tobytes()
    gathered = [None] * world
    dist.all_gather_object(gathered, (ms, cs))
    out[rank] = (t, gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_are_independent_and_time_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0][0] == 4.0 and res[1][0] == 4.0
    (ms0, cs0), (ms1, cs1) = res[0][1]
    assert ms0 != ms1 and cs0 != cs1
