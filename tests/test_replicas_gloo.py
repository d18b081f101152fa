"""The benchmark's multi-GPU path on CPU: replicas only (one filter step does
not shard without an exchange), two `gloo` ranks on 127.0.0.1.  Every rank
filters its own seeded workload, the job time is the slowest rank's, and the
job value counts every rank's steps."""

import json
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    t_local = (0.5, 0.8)[rank]  # rank 1 is the slower replica
    t_max = bench.max_over_ranks(t_local, world, device="cpu")
    value = bench.replica_value(10, t_max, world)
    seed = bench.replica_seed(rank)
    wl = synth.tomography_workload((16, 16), 4, 4, 2, 0.2, 1.0, 1e-4, seed=seed)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"{rank}.json"), "w") as f:
        json.dump({"t_max": t_max, "value": value, "seed": seed, "y0": wl["y"][0].tolist(),
                   "config": bench.bench_config(world)}, f)


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out = [json.load(open(tmp_path / f"{r}.json")) for r in range(world)]
    for o in out:
        assert o["t_max"] == 0.8  # the slowest rank's time, on every rank
        assert abs(o["value"] - world * 10 / 0.8) < 1e-12  # all ranks' steps / the job time
        assert o["config"]["global_batch"] == world and o["config"]["parallelism"] == "replicas x2"
    assert out[0]["seed"] != out[1]["seed"]
    assert not np.allclose(out[0]["y0"], out[1]["y0"])  # independent data per replica


def test_single_process_needs_no_collective():
    import bench

    assert bench.max_over_ranks(0.25, 1) == 0.25
    assert bench.replica_value(8, 0.5, 1) == 16.0
