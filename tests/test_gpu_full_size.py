"""Full-size workloads in the launch configuration the benchmark times, with
sampled elements compared against the FP64 oracle one by one (the oracle
integrates just the sampled elements)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1310_1194_gb300 import inputs
from parity_util import assert_grads_close, worst_conditioned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1310_1194_gb300 import api as a
    return a


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def sample(n, k, seed):
    """k element indices: the first, the last and k - 2 drawn at random."""
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=k - 2, replace=False)]))


def subset(w, idx):
    """The sampled elements as a workload of their own (per-point records by
    the points of each element)."""
    sub = {"geom": w["geom"][idx]}
    if w["per_qp"]:
        q = (np.asarray(w["degree"], dtype=np.int64) + 1) ** 3
        qo = np.concatenate([[0], np.cumsum(q)])
        rows = np.concatenate([np.arange(qo[e], qo[e + 1]) for e in idx])
    else:
        rows = idx
    for k in ("K", "b", "c", "f"):
        sub[k] = w[k][rows]
    return sub


def check(A, bv, st, w, idx, p, tol, Aoff=None, boff=None, degree=None):
    sub = subset(w, idx)
    deg = None if degree is None else np.asarray(degree)[idx]
    Ao, bo, so, (oA, ob, _) = oracle.integrate(sub["geom"], sub["K"], sub["b"], sub["c"], sub["f"],
                                               p=p, degree=deg, per_qp=w["per_qp"])
    stc = st.cpu().numpy()
    for j, e in enumerate(idx):
        s = oracle.nsh(p if deg is None else int(deg[j]))
        a0 = int(Aoff[e]) if Aoff is not None else int(e) * s * s
        b0 = int(boff[e]) if boff is not None else int(e) * s
        a = A[a0:a0 + s * s].double().cpu().numpy()
        b = bv[b0:b0 + s].double().cpu().numpy()
        ao = Ao[oA[j]:oA[j] + s * s]
        bb = bo[ob[j]:ob[j] + s]
        assert stc[e] == so[j]
        assert np.linalg.norm(a - ao) <= tol * np.linalg.norm(ao), (e, np.linalg.norm(a - ao) / np.linalg.norm(ao))
        assert np.linalg.norm(b - bb) <= tol * np.linalg.norm(bb), e


@pytest.mark.parametrize("name,k,tc", [("p4", 40, "tc_f16x3"), ("p7", 8, "tc_f16x3"), ("p1m", 64, "tc_f16x3"),
                                       ("p4", 16, "tc_3xtf32"), ("p7", 4, "tc_3xtf32")])
def test_uniform_workload_full_size(api, name, k, tc):
    w = inputs.workload(name)
    p = w["p"]
    prec = tc if p >= 3 else "fp32"
    g = [dev(w[x]) for x in ("geom", "K", "b", "c", "f")]
    refs = [api.fei_reference_create(p)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A, bv, st, _ = api.fei_integrate(*g, p=p, precision=prec, refs=refs)
    stream.synchronize()
    n = len(w["geom"])
    check(A, bv, st, w, sample(n, k, 11), p, 1e-6 if prec.startswith("tc") else 1e-5)


def test_mixed_workload_full_size_plan(api):
    """The 200 000-element mixed batch through a tuned plan (one graph)."""
    w = inputs.workload("mixed")
    deg = dev(w["degree"], torch.int32)
    g = [dev(w[x]) for x in ("geom", "K", "b", "c", "f")]
    layout = api.fei_plan_offsets(deg)
    plan = api.Plan(max_elem=len(w["geom"]), precision="tc_f16x3")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.tune(*g, degree=deg, layout=layout)
        A, bv, st, _ = plan.execute(*g, degree=deg, layout=layout)
    stream.synchronize()
    n = len(w["geom"])
    # six random elements of every degree, the first and the last
    rng = np.random.default_rng(12)
    degs = np.asarray(w["degree"])
    idx = np.unique(np.concatenate([[0, n - 1]] + [rng.choice(np.flatnonzero(degs == p), size=6, replace=False)
                                                   for p in range(1, 8)]))
    check(A, bv, st, w, idx, None, 1e-6, Aoff=layout.A_offset.cpu().numpy(), boff=layout.b_offset.cpu().numpy(),
          degree=w["degree"])


def test_diff_workload_full_size_forward_and_adjoint(api):
    """20 000 p = 5 elements with per-point fields: the forward and the
    quadratic-loss adjoint of the benchmark, sampled against the oracle's
    forward and adjoint."""
    w = inputs.workload("diff")
    p = w["p"]
    g = [dev(w[x]) for x in ("geom", "K", "b", "c", "f")]
    refs = [api.fei_reference_create(p)]
    n = len(w["geom"])
    s = oracle.nsh(p)
    u = inputs.loss_weights(n * s, 4)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A, bv, st, _ = api.fei_integrate(*g, p=p, per_qp=True, precision="tc_f16x3", refs=refs)
        grads = api.fei_integrate_backward_quadratic(*g, dev(u), p=p, per_qp=True, precision="fp32", refs=refs)
    stream.synchronize()
    idx = sample(n, 12, 13)
    check(A, bv, st, w, idx, p, 1e-6)
    sub = subset(w, idx)
    us = np.concatenate([u[e * s:(e + 1) * s] for e in idx])
    gA = np.concatenate([np.outer(us[j * s:(j + 1) * s], us[j * s:(j + 1) * s]).ravel() for j in range(len(idx))])
    ref = oracle.integrate_backward(sub["geom"], sub["K"], sub["b"], sub["c"], sub["f"], gA, -us, p=p,
                                    per_qp=True)
    q = (p + 1) ** 3
    rows = np.concatenate([np.arange(e * q, (e + 1) * q) for e in idx])
    got = [grads[0].cpu().numpy().reshape(n, 18)[idx]]
    got += [t.cpu().numpy().reshape(n * q, -1)[rows] for t in grads[1:]]
    # element by element and record by record (as in test_gpu_parity.py)
    assert_grads_close(got, ref, len(idx), True, np.full(len(idx), q), 1e-6, 1e-5, where="diff full size")


@pytest.mark.parametrize("precision,tol", [("tc_f16x3", 1e-6), ("fp64", 1e-12), ("fp32", 1e-5)])
def test_p7_worst_conditioned_elements(api, precision, tol):
    """The 32 768-prism p = 7 mesh (jitter 25 % of h): the 64 elements with
    the smallest det J over the quadrature points and the 64 with the largest
    ||J|| ||J^-1||, against the oracle element by element.  The split
    tensor-core path runs on the whole batch in the launch configuration the
    benchmark times; the FP64 and FP32 paths on the selected elements."""
    w = inputs.workload("p7")
    p = w["p"]
    idx = worst_conditioned(w["geom"], oracle.quadrature(p), k=64)
    assert len(idx) >= 64
    refs = [api.fei_reference_create(p)]
    if precision == "tc_f16x3":
        g = [dev(w[x]) for x in ("geom", "K", "b", "c", "f")]
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            A, bv, st, _ = api.fei_integrate(*g, p=p, precision=precision, refs=refs)
        stream.synchronize()
        check(A, bv, st, w, idx, p, tol)
    else:
        sub = subset(w, idx)
        g = [dev(sub[x]) for x in ("geom", "K", "b", "c", "f")]
        A, bv, st, _ = api.fei_integrate(*g, p=p, precision=precision, refs=refs)
        torch.cuda.synchronize()
        sw = dict(sub, per_qp=False)
        check(A, bv, st, sw, np.arange(len(idx)), p, tol)
