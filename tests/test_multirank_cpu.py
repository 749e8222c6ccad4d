"""The N > 1 host logic of bench.py on CPU with two gloo ranks: rank 0
compresses and writes the checkpoint, rank 1 imports it; both hold the same
compressed matrix, use different right-hand sides, and the whole-job value
divides all ranks' units by the slowest rank's time."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, tmpdir, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_1707_00164_b300 as G
    import workloads as wl
    w = wl.scaled(wl.C1, 800)
    K = w.matrix()
    h = bench.shared_handle(G, G.Entries.gaussian(K.points, w.bandwidth, w.shift),
                            G.default_params(leaf_size=32, max_rank=32), rank, world, dist.barrier,
                            os.path.join(tmpdir, "s.bin"))
    s = G.structure(h)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one

    def reduce_max(x):
        t = torch.tensor([x])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, ms_max = bench.whole_job_value(w.n, 16, world, ms, reduce_max)
    torch.save({"perm": s["perm"], "skel": [x.tolist() for x in s["skel"]], "value": value,
                "ms_max": ms_max, "seed": bench.rank_rhs_seed(w, rank)}, os.path.join(out, f"r{rank}.pt"))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_structure_and_aggregate(tmp_path):
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(2, port, str(tmp_path), str(tmp_path)), nprocs=2, join=True)
    r0 = torch.load(tmp_path / "r0.pt", weights_only=False)
    r1 = torch.load(tmp_path / "r1.pt", weights_only=False)
    assert np.array_equal(r0["perm"], r1["perm"]) and r0["skel"] == r1["skel"]
    assert r0["ms_max"] == r1["ms_max"] == 15.0
    assert r0["value"] == pytest.approx(800 * 16 * 2 / 0.015)
    assert r0["seed"] != r1["seed"]
