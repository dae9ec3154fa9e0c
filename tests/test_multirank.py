"""Probe sharding across ranks (one process per GPU) on CPU with gloo.

PICO's probes are independent (Alg. 1), so ``bench.py --gpus N`` gives each
rank a contiguous probe range (``shard_range``) and combines the partial
running sums with one all-reduce (``reduce_running_sums``, the product's own
exchange step).  Two checks with two gloo ranks:

* the product's shard-and-reduce path with a stub map producer: each rank
  fills its four running-sum maps (PICO sum / sumsq, PMR sum / sumsq) with
  per-sample contributions that depend only on the sample index, reduces them
  with ``reduce_running_sums``, and every rank must end with exactly the
  single-rank totals (integer-valued contributions: the sums are exact);
* the oracle's PICO sums over each shard, reduced the same way, equal a
  single-rank run over all probes (up to FP64 summation order).
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
    from paper_2605_09590_gb300 import reduce_running_sums, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S = synth.coil_maps(16, 12, 3, 1)
    op = O.Operator(S, None, mask=synth.mask_pe(16, 2, 2))
    begin, count = shard_range(total, world, rank)
    s, ss = OP.pico(op, 5, begin, count, 0.0, 20, 0.0)
    t = [torch.from_numpy(s), torch.from_numpy(ss)]
    reduce_running_sums(t)
    if rank == 0:
        np.save(out, np.stack([x.numpy() for x in t]))
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


def _stub_contribution(i, shape):
    """Per-sample map of sample i (integer valued, so every sum is exact)."""
    g = np.random.default_rng(1000 + i)
    return g.integers(-8, 9, size=shape).astype(np.float64)


def _stub_worker(rank, world, port, total, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2605_09590_gb300 import reduce_running_sums, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shape = (7, 5)
    maps = [torch.zeros(shape, dtype=torch.float64) for _ in range(4)]   # s, ss, ps, pss
    begin, count = shard_range(total, world, rank)
    for i in range(begin, begin + count):
        d = _stub_contribution(i, shape)
        p = _stub_contribution(10_000 + i, shape)
        maps[0] += torch.from_numpy(d)
        maps[1] += torch.from_numpy(d * d)
        maps[2] += torch.from_numpy(p)
        maps[3] += torch.from_numpy(p * p)
    reduce_running_sums(maps)
    np.save(out + f".{rank}.npy", np.stack([m.numpy() for m in maps]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,total", [(2, 13), (2, 1)])
def test_product_reduction_gives_every_rank_the_single_rank_totals(tmp_path, world, total):
    out = str(tmp_path / "maps")
    mp.start_processes(_stub_worker, args=(world, _free_port(), total, out), nprocs=world, start_method="spawn")
    shape = (7, 5)
    want = np.zeros((4,) + shape)
    for i in range(total):
        d = _stub_contribution(i, shape)
        p = _stub_contribution(10_000 + i, shape)
        want += np.stack([d, d * d, p, p * p])
    for r in range(world):
        got = np.load(out + f".{r}.npy")
        assert np.array_equal(got, want), r


def test_reduction_is_a_no_op_without_a_process_group():
    from paper_2605_09590_gb300 import reduce_running_sums
    t = [torch.ones(3, dtype=torch.float64)]
    reduce_running_sums(t)
    assert torch.equal(t[0], torch.ones(3, dtype=torch.float64))
