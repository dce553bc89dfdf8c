"""The N > 1 path on CPU: two gloo ranks, each taking its own kernel range the way
bench.py does (weak scaling, no data-path collective), with the slowest rank's time
reduced by MAX. The ranks' results put together equal one evaluation of the union,
which is what lets the path shard with no exchange."""

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, n, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from oracle import oracle as O
    from workloads import archs, gen

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = bench.shard(n, 2, "uneven", rank)
    r = O.evaluate(archs.arch("sm_103"), gen.axes(), d, 5)
    t = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
    dist.barrier()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), idx=r["idx"], cost=r["cost"], t=t,
             mask=d["space_mask"])
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange(tmp_path):
    from oracle import oracle as O
    from workloads import archs, gen

    world, n = 2, 300
    mp.start_processes(_rank, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert all(float(p["t"]) == 2.0 for p in parts)  # MAX over ranks, the same on every rank
    full_d = gen.descriptors(world * n, 2, "uneven")
    assert np.array_equal(np.concatenate([p["mask"] for p in parts]), full_d["space_mask"])  # disjoint, covering
    full = O.evaluate(archs.arch("sm_103"), gen.axes(), full_d, 5)
    assert np.array_equal(np.concatenate([p["idx"] for p in parts]), full["idx"])
    assert np.array_equal(np.concatenate([p["cost"] for p in parts]).view(np.uint32), full["cost"].view(np.uint32))
