"""Probe sharding across ranks (one process per GPU) on CPU with gloo.

PICO's probes are independent (Alg. 1), so ``bench.py --gpus N`` gives each
rank a contiguous probe range (``shard_range``) and combines the partial
running sums with one all-reduce.  Here two gloo ranks evaluate their shards
with the CPU oracle and the reduced map must equal a single-rank run over all
probes (up to FP64 summation order).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, total, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from oracle import ops as O
    from oracle import pico as OP
    from paper_2605_09590_gb300 import shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S = synth.coil_maps(16, 12, 3, 1)
    op = O.Operator(S, None, mask=synth.mask_pe(16, 2, 2))
    begin, count = shard_range(total, world, rank)
    s, ss = OP.pico(op, 5, begin, count, 0.0, 20, 0.0)
    t = torch.from_numpy(np.stack([s, ss]))
    dist.all_reduce(t)
    if rank == 0:
        np.save(out, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,total", [(2, 9), (2, 2)])
def test_sharded_probes_reduce_to_single_rank_map(tmp_path, world, total):
    import synth
    from oracle import ops as O
    from oracle import pico as OP

    out = str(tmp_path / "red.npy")
    mp.start_processes(_worker, args=(world, _free_port(), total, out), nprocs=world, start_method="spawn")
    got = np.load(out)
    S = synth.coil_maps(16, 12, 3, 1)
    op = O.Operator(S, None, mask=synth.mask_pe(16, 2, 2))
    s, ss = OP.pico(op, 5, 0, total, 0.0, 20, 0.0)
    assert np.allclose(got[0], s, rtol=1e-12, atol=1e-14)
    assert np.allclose(got[1], ss, rtol=1e-12, atol=1e-14)
