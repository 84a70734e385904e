"""The packed layout of host-memory batches (api.Pipeline.totals), without
a GPU: totals of N_sh^2, N_sh and per-point records against the offsets
the assembly oracle derives, and degrees outside 1..7 taking no room."""
import numpy as np
import pytest
import torch

from oracle import assembly as oas


@pytest.fixture(scope="module")
def Pipeline():
    from paper_1310_1194_gb300 import build
    build.build()
    from paper_1310_1194_gb300 import api
    return api.Pipeline


def test_uniform_totals(Pipeline):
    for p in range(1, 8):
        s = (p + 1) ** 2 * (p + 2) // 2
        assert Pipeline.totals(None, 10, p=p) == (10 * s * s, 10 * s, 10)
        assert Pipeline.totals(None, 10, p=p, per_qp=True) == (10 * s * s, 10 * s, 10 * (p + 1) ** 3)


def test_mixed_totals_and_bad_degrees(Pipeline):
    rng = np.random.default_rng(7)
    deg = rng.integers(1, 8, size=500).astype(np.int32)
    s, loff, moff = oas._offsets(deg)
    q = ((deg.astype(np.int64) + 1) ** 3).sum()
    assert Pipeline.totals(None, 500, degree=torch.from_numpy(deg), per_qp=True) == (moff[-1], loff[-1], q)
    assert Pipeline.totals(None, 500, degree=torch.from_numpy(deg))[2] == 500
    bad = deg.copy()
    bad[[3, 17]] = (0, 9)
    good = np.delete(deg, [3, 17])
    _, loff2, moff2 = oas._offsets(good)
    A_total, b_total, _ = Pipeline.totals(None, 500, degree=torch.from_numpy(bad))
    assert (A_total, b_total) == (moff2[-1], loff2[-1])
