"""The upper-triangle layout of A_e (FEI_A_UPPER) for a symmetric weak form
(b = 0, K symmetric: the Laplacian-type term of Sec. 2 plus reaction),
through the C ABI: against the oracle element by element, equal bit for bit
to the upper triangle of the full layout of the same path, non-symmetric
records flagged, and the same through plans and host-memory batches."""
import numpy as np
import pytest

import oracle
from paper_1310_1194_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tc_f16x3": 1e-6, "tc_3xtf32": 1e-6, "sf_fp32": 1e-5}


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_1194_gb300 import api as a
    return a


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def symmetric(w):
    """The workload with b = 0 and K replaced by (K + K^T) / 2 (exactly
    symmetric in FP64)."""
    K = np.asarray(w["K"]).reshape(-1, 3, 3)
    K = 0.5 * (K + np.swapaxes(K, 1, 2))
    return dict(w, K=np.ascontiguousarray(K.reshape(w["K"].shape)), b=np.zeros_like(w["b"]))


def triu_flat(A, p):
    s = oracle.nsh(p)
    iu = np.triu_indices(s)
    return A.reshape(-1, s, s)[:, iu[0], iu[1]].reshape(-1)


def run(api, w, p=None, degree=None, precision="fp64", per_qp=False, upper=False):
    A, bv, st, lay = api.fei_integrate(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                       p=p, degree=None if degree is None else dev(degree), per_qp=per_qp,
                                       precision=precision, upper=upper)
    torch.cuda.synchronize()
    return A.cpu().numpy(), bv.cpu().numpy(), st.cpu().numpy(), lay


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
@pytest.mark.parametrize("p", range(1, 8))
def test_upper_uniform_matches_oracle_and_full_layout(api, p, precision):
    n = {1: 300, 2: 90, 3: 40, 4: 21, 5: 9, 6: 5, 7: 3}[p]
    w = symmetric(inputs.workload("p7" if p >= 6 else "pr1", n_max=n))
    Au, bu, su, _ = run(api, w, p=p, precision=precision, upper=True)
    Af, bf, sf, _ = run(api, w, p=p, precision=precision)
    assert not su.any() and not sf.any()
    s = api.nsh(p)
    assert Au.size == n * s * (s + 1) // 2
    # the same accumulators, stored by the upper-layout path
    assert np.array_equal(Au.view(np.uint8), triu_flat(Af, p).view(np.uint8))
    assert np.array_equal(bu.view(np.uint8), bf.view(np.uint8))
    Ao, bo, so, _ = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], p=p)
    Ao3 = Ao.reshape(n, s, s)
    assert np.abs(Ao3 - np.swapaxes(Ao3, 1, 2)).max() <= 1e-13 * np.abs(Ao3).max()  # the oracle's A_e is symmetric
    ou = triu_flat(Ao, p).reshape(n, -1)
    gu = Au.astype(np.float64).reshape(n, -1)
    # relative Frobenius norm of the full matrix from its upper triangle
    diag = np.zeros(s * (s + 1) // 2, dtype=bool)
    diag[[i * s - i * (i - 1) // 2 for i in range(s)]] = True
    wgt = np.where(diag, 1.0, 2.0)
    err = np.sqrt((wgt * (gu - ou) ** 2).sum(1) / (wgt * ou ** 2).sum(1))
    assert err.max() < TOL[precision], err.max()
    full = api.unpack_upper(Au.reshape(n, -1), p)
    assert np.array_equal(np.triu(full[0]), np.triu(Af.reshape(n, s, s)[0]))


@pytest.mark.parametrize("precision", ["fp32", "tc_f16x3", "sf_fp32"])
def test_upper_mixed_batch_plan_and_per_point(api, precision):
    w = symmetric(inputs.workload("mixed", n_max=120))
    deg = w["degree"]
    Au, bu, su, lay = run(api, w, degree=deg, precision=precision, upper=True)
    Af, bf, sf, layf = run(api, w, degree=deg, precision=precision)
    assert not su.any()
    Aoff_u, Aoff_f = lay.A_offset.cpu().numpy(), layf.A_offset.cpu().numpy()
    for e in range(len(deg)):
        p = int(deg[e])
        s = api.nsh(p)
        full = Af[Aoff_f[e]:Aoff_f[e] + s * s]
        assert np.array_equal(Au[Aoff_u[e]:Aoff_u[e + 1]].view(np.uint8), triu_flat(full, p).view(np.uint8)), e
    # a plan (one graph) gives the same values
    plan = api.Plan(max_elem=len(deg), precision=precision)
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        Ap, bp, sp, _ = plan.execute(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                     degree=dev(deg), layout=lay, upper=True)
    s_.synchronize()
    assert np.array_equal(Ap.cpu().numpy().view(np.uint8), Au.view(np.uint8))
    # per-point symmetric fields at p = 5
    wd = inputs.workload("diff", n_max=4)
    q = 216
    Kq = np.broadcast_to(np.eye(3), (4 * q, 3, 3)) * (1.0 + 0.5 * np.sin(np.arange(4 * q)))[:, None, None]
    wd = dict(wd, K=np.ascontiguousarray(Kq), b=np.zeros((4 * q, 3)))
    Au, bu, su, _ = run(api, wd, p=5, precision=precision, per_qp=True, upper=True)
    Af, bf, sf, _ = run(api, wd, p=5, precision=precision, per_qp=True)
    assert not su.any() and np.array_equal(Au.view(np.uint8), triu_flat(Af, 5).view(np.uint8))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
@pytest.mark.parametrize("p", [1, 4, 7])
def test_upper_flags_records_that_are_not_symmetric(api, p, precision):
    w = symmetric(inputs.workload("p7" if p >= 6 else "pr1", n_max=6))
    K = w["K"].copy().reshape(-1, 9)
    K[1, 1] += 1e-3  # K01 != K10
    b = w["b"].copy()
    b[3, 2] = 0.25   # b != 0
    geom = w["geom"].copy()
    geom[4] = geom[4][[0, 2, 1, 3, 5, 4]]  # det J < 0 as well as b != 0 below
    b[4, 0] = 1.0
    w2 = dict(w, K=K.reshape(w["K"].shape), b=b, geom=geom)
    Au, bu, su, _ = run(api, w2, p=p, precision=precision, upper=True)
    assert list(su) == [0, 1, 0, 1, 3, 0]
    size = api.a_size(p, True)
    for e in (1, 3, 4):
        assert not Au[e * size:(e + 1) * size].any()
    # the full layout takes every element as given
    _, _, sf, _ = run(api, w2, p=p, precision=precision)
    assert list(sf) == [0, 0, 0, 0, 3, 0]


def test_upper_host_pipeline_equals_device(api):
    w = symmetric(inputs.workload("p4", n_max=900))
    p = 4
    Au, bu, su, _ = run(api, w, p=p, precision="tc_f16x3", upper=True)
    pipe = api.Pipeline(degrees=[p], precision="tc_f16x3", slot_bytes=1 << 20)
    h = {k: torch.from_numpy(np.ascontiguousarray(w[k])).pin_memory() for k in ("geom", "K", "b", "c", "f")}
    A, bv, st = pipe.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], p=p, upper=True)
    torch.cuda.synchronize()
    assert pipe.n_chunks > 1
    assert np.array_equal(A.numpy().view(np.uint8), Au.view(np.uint8))
    assert np.array_equal(bv.numpy().view(np.uint8), bu.view(np.uint8)) and not st.numpy().any()
