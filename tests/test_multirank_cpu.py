"""Tree sharding across ranks (gloo, world size 2, CPU): trees are indexed
globally, so ranks sampling disjoint tree ranges (shard.tree_range) and summing
R and C with one all-reduce (shard.allreduce_counts, the exchange the
multi-GPU benchmark runs) reproduce a single run exactly.  The samples come
from the CPU oracle sampler (the only sampler available without a GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import native
from paper_2101_06192_gb300 import shard

TAU = 40


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.barabasi_albert(400, 3, 8)
    first, count = shard.tree_range(rank, world, TAU)
    o = native.wilson(g, 1.0, seed=21, tau=count, tree_offset=first)
    R = torch.from_numpy(o["R"].astype(np.int64))
    C = torch.from_numpy(o["C"].astype(np.int64))
    shard.allreduce_counts(R, C)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # max-over-ranks timing reduction used by the bench
    if rank == 0:
        np.savez(out_path, R=R.numpy(), C=C.numpy(), tmax=t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_tree_sharding_matches_single_run(tmp_path):
    out = str(tmp_path / "r.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    g = synth.barabasi_albert(400, 3, 8)
    ref = native.wilson(g, 1.0, seed=21, tau=TAU)
    np.testing.assert_array_equal(got["R"], ref["R"].astype(np.int64))
    np.testing.assert_array_equal(got["C"], ref["C"].astype(np.int64))
    assert got["tmax"][0] == 2.0


def _rb_worker(rank, world, port, out_path):
    # Rao-Blackwellised totals are integers (fixed point), so ranks holding
    # disjoint tree ranges sum them exactly, in any order
    from oracle import rb
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.barabasi_albert(300, 3, 9)
    first, count = shard.tree_range(rank, world, 12)
    o = native.wilson(g, 0.7, seed=33, tau=count, tree_offset=first, want_parents=True)
    acc = torch.from_numpy(rb.accumulate(g, 0.7, o["parents"]).astype(np.int64))
    shard.allreduce_counts(acc)
    if rank == 0:
        np.save(out_path, acc.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_rao_blackwell_totals_match_single_run(tmp_path):
    from oracle import rb
    out = str(tmp_path / "acc.npy")
    mp.start_processes(_rb_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    g = synth.barabasi_albert(300, 3, 9)
    o = native.wilson(g, 0.7, seed=33, tau=12, want_parents=True)
    ref = rb.accumulate(g, 0.7, o["parents"]).astype(np.int64)
    np.testing.assert_array_equal(np.load(out), ref)


def test_tree_ranges_partition_the_trees():
    for tau in (0, 1, 7, 40, 1024):
        for world in (1, 2, 3, 8):
            spans = [shard.tree_range(r, world, tau) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == tau
            for (a, ca), (b, _) in zip(spans, spans[1:]):
                assert a + ca == b
    with pytest.raises(ValueError):
        shard.tree_range(2, 2, 10)
