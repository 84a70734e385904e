"""Host logic of bench.py on the CPU: the per-element error against the
oracle, and the sharding of a job over ranks (weak: translated copies of
the workload; strong: the workload itself), alone and as two gloo ranks
whose shards, integrated by the oracle and gathered, equal the whole job."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_1310_1194_gb300 import inputs, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_errors_vs_oracle_per_element():
    bench = load_bench()
    w = inputs.workload("mixed", n_max=30)
    ref = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], degree=w["degree"])
    Ao, bo, so, (oA, ob, _) = ref
    A = torch.from_numpy(Ao.astype(np.float32))
    bv = torch.from_numpy(bo.astype(np.float32))
    st = torch.from_numpy(so.copy())
    e = bench.errors_vs_oracle(A, bv, st, ref, 30)
    assert e["status_equal"] and e["elements"] == 30 and e["max"] < 1e-6 and e["b_max"] < 1e-6
    # one element made wrong by 1e-3 of its norm: its error shows, alone
    A2 = A.clone()
    k = 17
    sl = slice(int(oA[k]), int(oA[k + 1]))
    A2[sl] += torch.from_numpy(1e-3 * np.linalg.norm(Ao[sl]) / np.sqrt(oA[k + 1] - oA[k]) *
                               np.ones(int(oA[k + 1] - oA[k]))).float()
    e2 = bench.errors_vs_oracle(A2, bv, st, ref, 30)
    assert 0.9e-3 < e2["max"] < 1.1e-3 and e2["p99"] < 1e-3
    # a prefix of the batch only
    e3 = bench.errors_vs_oracle(A2, bv, st, ref, 10)
    assert e3["elements"] == 10 and e3["max"] < 1e-6


@pytest.mark.parametrize("name", ["p4", "mixed", "diff"])
def test_shards_cover_the_job(name):
    bench = load_bench()
    w = inputs.workload(name, n_max=90)
    n = len(w["geom"])
    for world in (1, 2, 3):
        strong = [bench.shard_workload(w, r, world, "strong") for r in range(world)]
        assert sum(len(s["geom"]) for s in strong) == n
        weak = [bench.shard_workload(w, r, world, "weak") for r in range(world)]
        assert sum(len(s["geom"]) for s in weak) == n * world
        if world > 1:
            # every element of the job exactly once, in job order; copy c
            # translated by c along x
            starts = [s["start"] for s in weak]
            assert starts == sorted(starts) and weak[0]["start"] == 0 and weak[-1]["end"] == n * world
            geom = np.concatenate([s["geom"] for s in weak])
            want = np.concatenate([w["geom"] + np.array([c, 0.0, 0.0]) for c in range(world)])
            np.testing.assert_array_equal(geom, want)
            deg = np.concatenate([s["degree"] for s in weak])
            np.testing.assert_array_equal(deg, np.tile(w["degree"], world))
            for k in ("K", "b", "c", "f"):
                np.testing.assert_array_equal(np.concatenate([s[k] for s in weak]),
                                              np.concatenate([w[k]] * world))
            # the split balances F(p): each rank within one element of its share
            F = shard.element_flops(deg)
            for s in weak:
                assert abs(F[s["start"]:s["end"]].sum() - F.sum() / world) <= F.max()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, mode, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = load_bench()
    w = inputs.workload("mixed", n_max=48)
    s = bench.shard_workload(w, rank, world, mode)
    A, bv, st, _ = oracle.integrate(s["geom"], s["K"], s["b"], s["c"], s["f"], degree=s["degree"])
    A, bv, st = shard.gather_outputs((torch.from_numpy(A), torch.from_numpy(bv), torch.from_numpy(st)))
    if rank == 0:
        np.savez(out_path, A=A.numpy(), b=bv.numpy(), st=st.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_gloo_ranks_integrate_the_job(tmp_path, mode):
    import torch.multiprocessing as mp
    out = str(tmp_path / "job.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), mode, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    w = inputs.workload("mixed", n_max=48)
    copies = 2 if mode == "weak" else 1
    geom = np.concatenate([w["geom"] + np.array([c, 0.0, 0.0]) for c in range(copies)])
    coef = {k: np.concatenate([w[k]] * copies) for k in ("K", "b", "c", "f")}
    A, bv, st, _ = oracle.integrate(geom, coef["K"], coef["b"], coef["c"], coef["f"],
                                    degree=np.tile(w["degree"], copies))
    np.testing.assert_array_equal(got["A"], A)
    np.testing.assert_array_equal(got["b"], bv)
    np.testing.assert_array_equal(got["st"], st)


def test_errors_vs_oracle_upper_layout():
    """A device result in the upper-triangle layout is mirrored back before
    the comparison: the oracle's own symmetric matrices, packed, give zero
    error; a change in one off-diagonal entry shows in its element only."""
    bench = load_bench()
    w = inputs.workload("p4sym", n_max=12)
    ref = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], p=4)
    Ao, bo, so, _ = ref
    s = 75
    iu = np.triu_indices(s)
    packed = Ao.reshape(12, s, s)[:, iu[0], iu[1]].reshape(-1)
    e = bench.errors_vs_oracle(torch.from_numpy(packed), torch.from_numpy(bo), torch.from_numpy(so), ref, 12,
                               upper_p=4)
    assert e["max"] < 1e-12, e
    bad = packed.copy()
    bad[5 * (s * (s + 1) // 2) + 3] += 1.0
    e = bench.errors_vs_oracle(torch.from_numpy(bad), torch.from_numpy(bo), torch.from_numpy(so), ref, 12,
                               upper_p=4)
    assert e["max"] > 1e-3 and e["p99"] > 1e-3 and e["mean"] < e["max"]


def test_unpack_upper_mirrors_the_triangle():
    from paper_1310_1194_gb300 import api
    rng = np.random.default_rng(0)
    M = rng.standard_normal((3, 18, 18))
    M = M + np.swapaxes(M, 1, 2)
    iu = np.triu_indices(18)
    packed = M[:, iu[0], iu[1]]
    assert packed.shape[-1] == api.a_size(2, True) == 171
    assert np.array_equal(api.unpack_upper(packed, 2), M)
    t = api.unpack_upper(torch.from_numpy(packed), 2)
    assert torch.equal(t, torch.from_numpy(M))
