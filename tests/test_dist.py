"""Host-side multi-rank logic of bench.py with two gloo ranks on CPU: rank discovery from
the environment, one independent pair per rank (weak scaling, no data-path collective),
barrier and the max-reduction of the step times."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist = bench.dist_init(w, "gloo")
    seed = bench.pair_seed(r)
    bench.barrier(dist)
    t = bench.reduce_max(1.0 + rank, dist)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{t} {' '.join(map(str, seeds))}")
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_shard_pairs(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        t, *seeds = open(tmp_path / f"r{rank}.txt").read().split()
        assert float(t) == 2.0                    # max over ranks
        assert seeds == ["0", "1"]                # each rank its own pair
    del torch


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.reduce_max(3.5, None) == 3.5
    bench.barrier(None)
