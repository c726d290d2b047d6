"""Multi-rank path on CPU (gloo, world size 2): each rank propagates its own
packet-id block and the int64 tallies are summed.  The reduced result must
equal a single-process run over all ids bit for bit.  The per-rank
propagation here uses the oracle (no GPU on this host); on GPUs each rank
launches the packet kernel on its block, and the exchange is the same
all-reduce of the same int64 tensors."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2112_08035_gb300.distributed import allreduce_tallies, shard_range


def test_shard_range_covers_ids_exactly():
    for n in (0, 1, 7, 1000, 10_000_001):
        for world in (1, 2, 3, 8):
            rs = [shard_range(r, world, n, base=5) for r in range(world)]
            assert rs[0][0] == 5 and rs[-1][1] == 5 + n
            for a, b in zip(rs, rs[1:]):
                assert a[1] == b[0]
            sizes = [e - b for b, e in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        import workloads as W
        wl = W.three_layer_slab(n, grid_n=24)
        b, e = shard_range(rank, world, n)
        flu, tot, _ = O.run(wl, b, e, threads=1)
        keys = ["R", "T", "A", "killed", "gain", "packets", "scatters", "steps"]
        f = torch.from_numpy(flu.copy())
        t = torch.tensor([tot[k] for k in keys], dtype=torch.int64)
        allreduce_tallies(f, t)
        if rank == 0:
            np.save(out + ".flu.npy", f.numpy())
            np.save(out + ".tot.npy", t.numpy())
    finally:
        torch.distributed.destroy_process_group()


@pytest.mark.parametrize("n", [301, 1000])
def test_two_rank_allreduce_equals_single_run(tmp_path, n):
    import oracle as O
    import workloads as W
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(2, _free_port(), n, out), nprocs=2, join=True, start_method="spawn")
    flu = np.load(out + ".flu.npy")
    tot = np.load(out + ".tot.npy")
    f1, t1, _ = O.run(W.three_layer_slab(n, grid_n=24), 0, n, threads=1)
    keys = ["R", "T", "A", "killed", "gain", "packets", "scatters", "steps"]
    assert np.array_equal(flu, f1)
    assert list(tot) == [t1[k] for k in keys]
