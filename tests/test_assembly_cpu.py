"""Assembly (Sec. 2) without a GPU: the assembly oracle against what fixes
it (a hand example, brute force, the block-diagonal case, quadratic-form and
row-sum identities), and the library's host part (pattern, colouring,
argument checks) in host-only mode against the oracle."""
import numpy as np
import pytest

from oracle import assembly as oas
from paper_1310_1194_gb300 import inputs


def nsh(p):
    return (p + 1) ** 2 * (p + 2) // 2


def random_blocks(degrees, seed):
    rng = np.random.default_rng(seed)
    s = np.array([nsh(int(p)) for p in degrees])
    A = rng.standard_normal(int((s * s).sum()))
    b = rng.standard_normal(int(s.sum()))
    return A, b


def test_hand_example_two_elements_sharing_three_functions():
    """Two p = 1 elements (6 functions each) sharing global functions 3, 4, 5:
    the overlap block of K is the sum of the two corner blocks, the rest are
    copies, and rhs adds the shared entries."""
    A0 = np.arange(36, dtype=float).reshape(6, 6)
    A1 = 100.0 + np.arange(36, dtype=float).reshape(6, 6)
    l2g = np.array([0, 1, 2, 3, 4, 5, 3, 4, 5, 6, 7, 8])
    b = np.arange(12, dtype=float)
    K = np.zeros((9, 9))
    K[:6, :6] += A0
    K[3:9, 3:9] += A1
    rhs = np.zeros(9)
    rhs[:6] += b[:6]
    rhs[3:] += b[6:]
    rp, ci, v, r = oas.assemble(np.concatenate([A0.ravel(), A1.ravel()]), b, l2g, 9, [1, 1])
    assert np.array_equal(oas.csr_to_dense(rp, ci, v, 9), K)
    assert np.array_equal(r, rhs)
    # the pattern lists exactly the nonzero blocks
    assert list(rp) == [0, 6, 12, 18, 27, 36, 45, 51, 57, 63]
    assert list(ci[18:27]) == list(range(9))


def test_assemble_matches_the_plain_loop():
    w = inputs.workload("mixed", n_max=40)
    l2g, nd = inputs.dof_map(w)
    A, b = random_blocks(w["degree"], 1)
    rp, ci, v, r = oas.assemble(A, b, l2g, nd, w["degree"])
    K, rhs = oas.assemble_dense(A, b, l2g, nd, w["degree"])
    assert np.allclose(oas.csr_to_dense(rp, ci, v, nd), K, rtol=1e-14, atol=1e-13)
    assert np.allclose(r, rhs, rtol=1e-14, atol=1e-13)
    # the stored entries are exactly those that receive a contribution
    hit = oas.assemble_dense(np.ones_like(A), b, l2g, nd, w["degree"])[0]
    assert np.array_equal(np.flatnonzero(oas.csr_to_dense(rp, ci, np.ones_like(v), nd)), np.flatnonzero(hit))


def test_pins_catch_planted_mistakes(monkeypatch):
    """The hand example fails for an oracle that swaps row and column, and
    for one that stores instead of adding."""
    A0 = np.arange(36, dtype=float)
    A1 = 100.0 + np.arange(36, dtype=float)
    A = np.concatenate([A0, A1])
    l2g = np.array([0, 1, 2, 3, 4, 5, 3, 4, 5, 6, 7, 8])
    b = np.arange(12, dtype=float)
    K, _ = oas.assemble_dense(A, b, l2g, 9, [1, 1])
    good = oas.csr_to_dense(*oas.assemble(A, b, l2g, 9, [1, 1])[:3], 9)
    assert np.array_equal(good, K)
    real_repeat, real_tile = np.repeat, np.tile
    monkeypatch.setattr(oas.np, "repeat", real_tile)   # rows and columns swapped
    monkeypatch.setattr(oas.np, "tile", real_repeat)
    swapped = oas.csr_to_dense(*oas.assemble(A, b, l2g, 9, [1, 1])[:3], 9)
    monkeypatch.undo()
    assert not np.array_equal(swapped, K)

    def store(a, idx, v):  # assignment keeps one contribution per entry
        a[idx] = v
    monkeypatch.setattr(oas.np.add, "at", store, raising=False)
    stored = oas.csr_to_dense(*oas.assemble(A, b, l2g, 9, [1, 1])[:3], 9)
    monkeypatch.undo()
    assert not np.array_equal(stored, K)


def test_private_numbering_gives_the_block_diagonal():
    w = inputs.workload("mixed", n_max=30)
    l2g, nd = inputs.dof_map(w, shared="none")
    A, b = random_blocks(w["degree"], 2)
    rp, ci, v, r = oas.assemble(A, b, l2g, nd, w["degree"])
    s = np.array([nsh(int(p)) for p in w["degree"]])
    assert np.array_equal(v, A)  # each row is one element row, in order
    assert np.array_equal(r, b)
    assert np.array_equal(np.diff(rp), np.repeat(s, s))


def test_quadratic_form_and_row_sums():
    """u^T K u = sum_e u_e^T A_e u_e and K 1 = gather of A_e 1."""
    w = inputs.workload("pr1", n_max=200)
    l2g, nd = inputs.dof_map(w)
    A, b = random_blocks(w["degree"], 3)
    rp, ci, v, r = oas.assemble(A, b, l2g, nd, w["degree"])
    u = np.random.default_rng(4).standard_normal(nd)
    Ku = np.zeros(nd)
    for row in range(nd):
        Ku[row] = v[rp[row]:rp[row + 1]] @ u[ci[rp[row]:rp[row + 1]]]
    q = 0.0
    rs = np.zeros(nd)
    for e in range(len(w["degree"])):
        g = l2g[6 * e:6 * e + 6]
        Ae = A[36 * e:36 * e + 36].reshape(6, 6)
        q += u[g] @ Ae @ u[g]
        np.add.at(rs, g, Ae.sum(axis=1))
    assert abs(u @ Ku - q) <= 1e-12 * np.abs(A).sum()
    Kones = np.array([v[rp[row]:rp[row + 1]].sum() for row in range(nd)])
    assert np.allclose(Kones, rs, rtol=1e-13, atol=1e-12)


@pytest.fixture(scope="module")
def api():
    from paper_1310_1194_gb300 import build
    build.build()
    from paper_1310_1194_gb300 import api as a
    return a


@pytest.mark.parametrize("name,n", [("pr1", 300), ("mixed", 150), ("p4", 40)])
def test_host_pattern_matches_the_oracle(api, name, n):
    w = inputs.workload(name, n_max=n)
    l2g, nd = inputs.dof_map(w)
    deg = w["degree"] if w["p"] is None else None
    asm = api.Assembly(l2g, nd, p=w["p"], degree=deg, host_only=True)
    rp, ci, colour = asm.pattern()
    A, b = random_blocks(w["degree"], 5)
    orp, oci, _, _ = oas.assemble(A, b, l2g, nd, w["degree"])
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    assert asm.nnz == len(oci) and asm.n_dof == nd


@pytest.mark.parametrize("name,n", [("pr1", 500), ("mixed", 300)])
def test_colouring_separates_elements_that_share_a_function(api, name, n):
    w = inputs.workload(name, n_max=n)
    l2g, nd = inputs.dof_map(w)
    deg = w["degree"] if w["p"] is None else None
    asm = api.Assembly(l2g, nd, p=w["p"], degree=deg, host_only=True)
    _, _, colour = asm.pattern()
    s = np.array([nsh(int(p)) for p in w["degree"]])
    off = np.concatenate([[0], np.cumsum(s)])
    owner = {}
    for e in range(len(s)):
        for d in l2g[off[e]:off[e + 1]]:
            owner.setdefault(int(d), []).append(e)
    most = 0
    for es in owner.values():
        cs = [colour[e] for e in es]
        assert len(set(cs)) == len(cs)  # no colour twice around one function
        most = max(most, len(es))
    assert asm.n_colours >= most and colour.min() == 0 and colour.max() == asm.n_colours - 1


def test_host_argument_errors(api):
    from paper_1310_1194_gb300._lib import FeiError
    l2g = np.array([0, 1, 2, 3, 4, 5], dtype=np.int64)
    with pytest.raises(FeiError, match="outside"):
        api.Assembly(l2g, 5, p=1, host_only=True)
    with pytest.raises(FeiError, match="twice"):
        api.Assembly(np.array([0, 1, 2, 3, 4, 4]), 6, p=1, host_only=True)
    with pytest.raises(FeiError):
        api.Assembly(l2g, 6, degree=np.array([9], dtype=np.int32), host_only=True)
