"""The multi-rank path on the CPU: two gloo ranks each sample their tree
range (the oracle's sequential Wilson on the same Philox stacks), add their
visit sums with the all-reduce of ``shard.all_reduce_sums``, and must equal
one process sampling both ranges, bit for bit."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import wilson as ow
from paper_2510_20604_gb300 import shard

T = 24


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.ba(300, 3, seed=5)
        smp = ow.Sampler(g, root=int(np.argmax(np.diff(g.row_ptr))), seed=11)
        t0, cnt = shard.tree_range(rank, world, T, tree0=1000)
        sums = torch.tensor(smp.sample(t0, cnt)["sums"], dtype=torch.float64)
        shard.all_reduce_sums(sums)
        if rank == 0:
            np.save(out, sums.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_equal_one_process(world):
    out = os.path.join(tempfile.mkdtemp(), "sums.npy")
    mp.start_processes(_rank, args=(world, _port(), out), nprocs=world, start_method="spawn", join=True)
    got = np.load(out)
    g = synth.ba(300, 3, seed=5)
    smp = ow.Sampler(g, root=int(np.argmax(np.diff(g.row_ptr))), seed=11)
    want = smp.sample(1000, world * T)["sums"]
    assert np.array_equal(got, want)


def test_tree_range():
    assert shard.tree_range(0, 4, 500) == (0, 500)
    assert shard.tree_range(3, 4, 500, tree0=7) == (1507, 500)
    with pytest.raises(ValueError):
        shard.tree_range(4, 4, 500)
    with pytest.raises(ValueError):
        shard.tree_range(1, 2, 1 << 31, tree0=1)
