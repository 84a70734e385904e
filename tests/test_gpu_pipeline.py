"""Host-memory batches (fei_integrate_host): inputs and outputs in host
memory, cut into chunks that pass through two device slots.  The element
matrices must be those of fei_integrate bit for bit (same kernels on the
same elements), in the packed layout, whatever the chunking; statuses
likewise; and sampled elements agree with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1310_1194_gb300 import inputs

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture(scope="module")
def api():
    from paper_1310_1194_gb300 import api as a
    return a


def host(w, pinned=True):
    t = {k: torch.from_numpy(np.ascontiguousarray(w[k])) for k in ("geom", "K", "b", "c", "f")}
    return {k: (v.pin_memory() if pinned else v) for k, v in t.items()}


def packed_layout(api, deg):
    """The packed layout with degrees outside 1..7 taking no room (the
    Python fei_plan_offsets refuses such degrees)."""
    d = np.asarray(deg, dtype=np.int64)
    ok = (d >= 1) & (d <= 7)
    s = np.where(ok, (d + 1) ** 2 * (d + 2) // 2, 0)
    q = np.where(ok, (d + 1) ** 3, 0)
    off = [np.concatenate([[0], np.cumsum(x)]) for x in (s * s, s, q)]
    return api.Layout(*[torch.from_numpy(o).cuda() for o in off], *[int(o[-1]) for o in off])


def device_reference(api, w, precision, refs, degree=None, layout=None):
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    if degree is None:
        A, bv, st, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=w["p"], per_qp=w["per_qp"],
                                         precision=precision, refs=refs)
    else:
        d = torch.from_numpy(np.ascontiguousarray(degree)).to(torch.int32).cuda()
        A, bv, st, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=d,
                                         per_qp=w["per_qp"], precision=precision, refs=refs, layout=layout)
    torch.cuda.synchronize()
    return A.cpu(), bv.cpu(), st.cpu()


@pytest.mark.parametrize("name,n,precision,slot", [("p4", 3001, "tc_f16x3", MIB), ("p4", 500, "fp64", 0),
                                                    ("p1m", 20000, "fp32", MIB), ("p7", 9, "tc_f16x3", MIB)])
def test_uniform_equals_device_path(api, name, n, precision, slot):
    w = inputs.workload(name, n_max=n)
    p = w["p"]
    refs = [api.fei_reference_create(p)]
    pl = api.Pipeline(precision=precision, slot_bytes=slot, refs=refs)
    h = host(w)
    A, bv, st = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], p=p)
    torch.cuda.current_stream().synchronize()
    if slot:
        assert pl.n_chunks > 1
    Ad, bd, sd = device_reference(api, w, precision, refs)
    assert torch.equal(A, Ad) and torch.equal(bv, bd) and torch.equal(st, sd)
    assert int(st.abs().max()) == 0


@pytest.mark.parametrize("precision,tol", [("tc_f16x3", 1e-6), ("fp64", 1e-12)])
def test_mixed_against_device_path_and_oracle(api, precision, tol):
    w = inputs.workload("mixed", n_max=900)
    refs = [api.fei_reference_create(d) for d in range(1, 8)]
    pl = api.Pipeline(precision=precision, slot_bytes=2 * MIB, refs=refs)
    h = host(w)
    deg = torch.from_numpy(np.ascontiguousarray(w["degree"])).to(torch.int32)
    A, bv, st = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], degree=deg)
    torch.cuda.current_stream().synchronize()
    assert pl.n_chunks > 2
    Ad, bd, sd = device_reference(api, w, precision, refs, degree=w["degree"])
    assert torch.equal(A, Ad) and torch.equal(bv, bd) and torch.equal(st, sd)
    idx = np.arange(0, len(w["degree"]), 37)
    Ao, bo, so, (oA, ob, _) = oracle.integrate(w["geom"][idx], w["K"][idx], w["b"][idx], w["c"][idx], w["f"][idx],
                                               degree=w["degree"][idx])
    s = (w["degree"].astype(np.int64) + 1) ** 2 * (w["degree"].astype(np.int64) + 2) // 2
    aoff = np.concatenate([[0], np.cumsum(s * s)])
    for j, e in enumerate(idx):
        got = A[aoff[e]:aoff[e + 1]].double().numpy()
        want = Ao[oA[j]:oA[j] + s[e] ** 2]
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), e


def test_per_point_coefficients_and_pageable_memory(api):
    """Per-point records (p = 5) chunked by records, from pageable host
    tensors into pageable outputs."""
    w = inputs.workload("diff", n_max=40)
    refs = [api.fei_reference_create(5)]
    pl = api.Pipeline(precision="tc_f16x3", slot_bytes=MIB, refs=refs)
    h = host(w, pinned=False)
    s = 126
    out = (torch.empty(40 * s * s), torch.empty(40 * s), torch.empty(40, dtype=torch.int32))
    A, bv, st = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], p=5, per_qp=True, out=out)
    torch.cuda.current_stream().synchronize()
    assert pl.n_chunks > 1 and A is out[0]
    Ad, bd, sd = device_reference(api, w, "tc_f16x3", refs)
    assert torch.equal(A, Ad) and torch.equal(bv, bd) and torch.equal(st, sd)


def test_flags_and_bad_degree_and_reuse(api):
    """An inverted prism and an element of degree 9 are flagged as by
    fei_integrate (the bad degree takes no room in the packed layout), and a
    second batch through the same pipeline (slots reused across calls)
    still matches."""
    w = dict(inputs.workload("mixed", n_max=300))
    geom = w["geom"].copy()
    geom[4] = geom[4][[0, 2, 1, 3, 5, 4]]
    w["geom"] = geom
    deg = w["degree"].copy()
    deg[11] = 9
    refs = [api.fei_reference_create(d) for d in range(1, 8)]
    pl = api.Pipeline(precision="fp32", slot_bytes=MIB, refs=refs)
    h = host(w)
    A, bv, st = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], degree=torch.from_numpy(deg).to(torch.int32))
    torch.cuda.current_stream().synchronize()
    Ad, bd, sd = device_reference(api, w, "fp32", refs, degree=deg, layout=packed_layout(api, deg))
    assert torch.equal(st, sd) and int(st[4]) != 0 and int(st[11]) == 2
    ok = np.flatnonzero(sd.numpy() == 0)
    s = np.where((deg >= 1) & (deg <= 7), (deg.astype(np.int64) + 1) ** 2 * (deg.astype(np.int64) + 2) // 2, 0)
    aoff = np.concatenate([[0], np.cumsum(s * s)])
    for e in ok:
        assert torch.equal(A[aoff[e]:aoff[e + 1]], Ad[aoff[e]:aoff[e + 1]])
    w2 = inputs.workload("p4", n_max=120)
    h2 = host(w2)
    A2, b2, st2 = pl.integrate_host(h2["geom"], h2["K"], h2["b"], h2["c"], h2["f"], p=4)
    torch.cuda.current_stream().synchronize()
    Ad2, bd2, _ = device_reference(api, w2, "fp32", refs)
    assert torch.equal(A2, Ad2) and torch.equal(b2, bd2)


def test_refused_arguments(api):
    from paper_1310_1194_gb300._lib import FeiError
    refs = [api.fei_reference_create(4)]
    with pytest.raises(FeiError, match="slot_bytes"):
        api.Pipeline(precision="fp32", slot_bytes=1000, refs=refs)
    pl = api.Pipeline(precision="fp32", slot_bytes=MIB, refs=refs)
    w = inputs.workload("p4", n_max=8)
    h = host(w)
    with pytest.raises(ValueError, match="host"):
        pl.integrate_host(h["geom"].cuda(), h["K"], h["b"], h["c"], h["f"], p=4)
    with pytest.raises(ValueError, match="K must hold"):
        pl.integrate_host(h["geom"], h["K"].reshape(-1)[:9], h["b"], h["c"], h["f"], p=4)
    # a degree with no reference in the pipeline: flagged, not integrated
    deg = torch.full((8,), 4, dtype=torch.int32)
    deg[3] = 5
    A, bv, st = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], degree=deg)
    torch.cuda.current_stream().synchronize()
    assert int(st[3]) == 2 and int(st.abs().sum()) == 2


def test_pipeline_scratch_is_its_own(api):
    """A mixed batch through the pipeline on one stream while fei_integrate
    integrates another mixed batch on a second stream: both results are
    right (the pipeline buckets degrees in its own scratch, not in the
    workspace that fei_integrate keeps per device)."""
    w1 = inputs.workload("mixed", n_max=700)
    w2 = dict(inputs.workload("mixed", n_max=900))
    w2["geom"] = w2["geom"] * 1.5  # a different batch
    refs = [api.fei_reference_create(d) for d in range(1, 8)]
    A1r, b1r, _ = device_reference(api, w1, "fp32", refs, degree=w1["degree"])
    A2r, b2r, _ = device_reference(api, w2, "fp32", refs, degree=w2["degree"])
    pl = api.Pipeline(precision="fp32", slot_bytes=MIB, refs=refs)
    h = host(w1)
    hdeg = torch.from_numpy(np.ascontiguousarray(w1["degree"])).to(torch.int32).pin_memory()
    g2 = {k: torch.from_numpy(np.ascontiguousarray(w2[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    d2 = torch.from_numpy(np.ascontiguousarray(w2["degree"])).to(torch.int32).cuda()
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        A1, b1, st1 = pl.integrate_host(h["geom"], h["K"], h["b"], h["c"], h["f"], degree=hdeg)
    with torch.cuda.stream(s2):
        for _ in range(3):
            A2, b2, st2, _ = api.fei_integrate(g2["geom"], g2["K"], g2["b"], g2["c"], g2["f"], degree=d2,
                                               precision="fp32", refs=refs)
    torch.cuda.synchronize()
    assert pl.n_chunks > 2
    assert torch.equal(A1, A1r) and torch.equal(b1, b1r)
    assert torch.equal(A2.cpu(), A2r) and torch.equal(b2.cpu(), b2r)
