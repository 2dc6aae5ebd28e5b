"""The multi-rank path of the benchmark on CPU (gloo, world size 2): each rank takes its own slice
of the seeded stream (no data exchange between ranks), and the job's time is the slowest rank's
(the one collective).  No GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import gcngen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank, out_dir):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first = bench.rank_first(rank, per_rank)
        b = gcngen.generate(1, per_rank, seed=gcngen.SEED_BASE + 1, first=first, threads=1)
        np.save(os.path.join(out_dir, f"text{rank}.npy"), b.text)
        np.save(os.path.join(out_dir, f"off{rank}.npy"), b.offsets)
        my_ms = 10.0 + 5.0 * rank  # a stand-in for this rank's measured time
        slowest = bench.max_over_ranks(torch, my_ms, "cpu")
        with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as f:
            f.write(repr(slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_disjoint_slices_and_the_slowest_time(tmp_path):
    if not dist.is_available() or not dist.is_gloo_available():
        pytest.skip("torch.distributed with gloo is not available")
    per_rank = 6
    mp.start_processes(_rank_main, args=(2, _free_port(), per_rank, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    whole = gcngen.generate(1, 2 * per_rank, seed=gcngen.SEED_BASE + 1, threads=1)
    kernels = []
    for r in range(2):
        text = np.load(tmp_path / f"text{r}.npy")
        off = np.load(tmp_path / f"off{r}.npy")
        kernels += [text[off[i]:off[i + 1]].tobytes() for i in range(per_rank)]
        assert float(open(tmp_path / f"max{r}.txt").read()) == 15.0
    # the two slices are the first 2 * per_rank kernels of the stream, in order, none twice
    assert kernels == [whole.kernel(i) for i in range(2 * per_rank)]
    assert len(set(kernels)) == len(kernels)
