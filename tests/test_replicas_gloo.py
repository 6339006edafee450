"""The multi-GPU path of bench.py is replicas only: each rank takes its own
sources and the job's rate is all queries over the slowest rank's time.  This
runs that logic as two gloo ranks on the CPU (no GPU, no collective on the data
path)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    w = dict(bench.WORKLOADS["cl100k"])
    n, rp, col = synth.chung_lu(3000, 20000, gamma=2.1, seed=1)
    srcs = bench.sources_for(w, rp, world, rank)
    per_rank_ms = 100.0 * (rank + 1)  # rank 1 is the slowest
    total_ms, other = bench.reduce_max([per_rank_ms, float(rank)], "cpu")
    rate = bench.whole_job_rate(len(srcs), world, total_ms)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([total_ms, other, rate] + list(srcs), dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 200.0          # max over ranks
    assert r0[1] == r1[1] == 1.0
    # rank r takes entries [10 r, 10 r + 10) of one seeded list of 20 sources
    sys.path.insert(0, ROOT)
    import synth
    n, rp, col = synth.chung_lu(3000, 20000, gamma=2.1, seed=1)
    allsrc = synth.random_sources(rp, 20, seed=7)
    assert np.array_equal(r0[3:].astype(int), allsrc[:10])
    assert np.array_equal(r1[3:].astype(int), allsrc[10:])
    assert r0[2] == pytest.approx(20 / 0.2)  # 20 queries over the slowest rank's 0.2 s
