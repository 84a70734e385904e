"""Sharding over ranks (paper_1310_1194_gb300/shard.py): contiguous element
ranges balanced by the algorithmic work F(p), and a two-rank gloo run on CPU
whose per-rank results, gathered, equal the single-process batch bit for
bit (elements are independent, Sec. 2)."""
import os
import socket

import numpy as np
import pytest

from paper_1310_1194_gb300 import inputs, shard


def test_partition_covers_and_balances():
    deg = inputs.mixed_degrees(5000, 3)
    F = shard.element_flops(deg)
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition(deg, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(deg)
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
        ideal = F.sum() / world
        for a, b in parts:
            # each range is within one element's work of the ideal share
            assert abs(F[a:b].sum() - ideal) <= F.max() * 1.0001
    assert shard.partition(np.zeros(0, dtype=np.int32), 3) == [(0, 0)] * 3
    # uniform degree: equal counts up to one element
    parts = shard.partition(np.full(1001, 4), 4)
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1


def test_element_flops_matches_the_paper_convention():
    # F(p) = 8 N_sh^2 N_q + 2 N_sh N_q + 220 N_q
    assert shard.element_flops([4])[0] == 8 * 75 * 75 * 125 + 2 * 75 * 125 + 220 * 125
    assert shard.element_flops([1])[0] == 8 * 36 * 8 + 2 * 6 * 8 + 220 * 8


def test_shard_slices_per_point_coefficients():
    w = inputs.workload("diff", n_max=40)
    parts = [shard.shard(w, r, 3) for r in range(3)]
    assert sum(len(s["geom"]) for s in parts) == 40
    q = 6 ** 3
    for s in parts:
        n = len(s["geom"])
        assert s["K"].shape[0] == n * q and s["c"].shape[0] == n * q
        np.testing.assert_array_equal(s["K"], w["K"][s["start"] * q:s["end"] * q])


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = inputs.workload("mixed", n_max=240)
    s = shard.shard(w, rank, world)
    A, bv, st, _ = oracle.integrate(s["geom"], s["K"], s["b"], s["c"], s["f"], degree=s["degree"], nthreads=1)
    A_all, b_all, st_all = shard.gather_outputs((torch.from_numpy(A), torch.from_numpy(bv), torch.from_numpy(st)))
    if rank == 0:
        np.savez(out_path, A=A_all.numpy(), b=b_all.numpy(), st=st_all.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_concatenate_bitwise(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    out = str(tmp_path / "gathered.npz")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w = inputs.workload("mixed", n_max=240)
    A, bv, st, _ = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], degree=w["degree"], nthreads=1)
    assert np.array_equal(got["A"], A)
    assert np.array_equal(got["b"], bv)
    assert np.array_equal(got["st"], st)
