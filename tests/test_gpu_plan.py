"""Plans (include/fei.h): a mixed-degree batch captured into a CUDA graph,
with per-degree kernel shapes chosen by the autotuner.  Results must agree
with fei_integrate and with the FP64 oracle, stay identical across graph
replays, and survive a re-capture with new output buffers."""
import numpy as np
import pytest

import oracle
from paper_1310_1194_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


def _mixed(n, seed_name="mixed"):
    w = inputs.workload(seed_name, n_max=n)
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    deg = torch.from_numpy(np.ascontiguousarray(w["degree"])).cuda()
    return w, g, deg


@pytest.mark.parametrize("precision,tol", [("tc_f16x3", 1e-6), ("fp32", 1e-5), ("fp64", 1e-12), ("sf_fp32", 1e-5),
                                           ("auto", 1e-6)])
def test_plan_matches_integrate_and_oracle(precision, tol):
    from paper_1310_1194_gb300 import api
    w, g, deg = _mixed(700)
    n = g["geom"].shape[0]
    layout = api.fei_plan_offsets(deg)
    plan = api.Plan(max_elem=n, precision=precision)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A, bv, st, _ = plan.tune(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout)
        A1, b1, st1, _ = plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout)
        A1c, b1c = A1.clone(), b1.clone()
        # replay of the captured graph into the same buffers
        plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout, out=(A1, b1, st1))
        Ar, br, str_, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg,
                                            precision=precision, layout=layout)
    s.synchronize()
    assert int(st1.abs().max()) == 0
    assert torch.equal(A1, A1c) and torch.equal(b1, b1c)
    Ao, bo, sto, off = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], degree=w["degree"])
    assert int(np.abs(sto).max()) == 0
    Ah, bh = A1.double().cpu().numpy(), b1.double().cpu().numpy()
    Arh = Ar.double().cpu().numpy()
    Aoff = layout.A_offset.cpu().numpy()
    for e in range(n):
        sl = slice(int(Aoff[e]), int(Aoff[e + 1]))
        assert _rel(Ah[sl], Ao[sl]) <= tol, (e, int(w["degree"][e]))
        assert _rel(Ah[sl], Arh[sl]) <= tol
    boff = layout.b_offset.cpu().numpy()
    for e in range(0, n, 7):
        sl = slice(int(boff[e]), int(boff[e + 1]))
        assert np.linalg.norm(bh[sl] - bo[sl]) <= tol * max(np.linalg.norm(bo[sl]), 1e-14) + 1e-12
    for p in range(1, 8):
        v, cap, ms = plan.choice(p)
        assert v >= 0 and cap >= 0
        if (w["degree"] == p).any():
            assert ms > 0.0
        kernel = plan.kernel(p)
        if p <= 2 or precision in ("fp32", "fp64"):
            assert kernel == "cuda_core"
        elif precision == "auto":
            assert kernel in ("tensor_core", "sum_factorised")
        else:
            assert kernel == {"tc_f16x3": "tensor_core", "sf_fp32": "sum_factorised"}[precision]


def test_auto_precision_resolves_per_degree():
    """FEI_AUTO on a direct call runs FEI_FP32 at p <= 2, FEI_TC_F16X3 at
    p = 3, 4 and the sum-factorised kernel at p = 5..7: bit for bit the
    outputs of those precisions.  Under a plan, a tensor-core variant or the
    sum-factorised variant (number = the tensor-core variant count) can be
    chosen by hand."""
    from paper_1310_1194_gb300 import api, _lib
    for p, same in ((1, "fp32"), (3, "tc_f16x3"), (4, "tc_f16x3"), (5, "sf_fp32"), (6, "sf_fp32"), (7, "sf_fp32")):
        w = inputs.workload("p7" if p >= 6 else "pr1", n_max=40 if p >= 6 else 300)
        g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
        Aa, ba, sa, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=p, precision="auto")
        As, bs, ss, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=p, precision=same)
        torch.cuda.synchronize()
        assert torch.equal(Aa, As) and torch.equal(ba, bs) and torch.equal(sa, ss), (p, same)
    n = 40
    w = inputs.workload("p7", n_max=n)
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    plan = api.Plan(degrees=[5], max_elem=n, precision="auto")
    assert plan.kernel(5) == "sum_factorised"
    plan.set_choice(5, 0, 0)
    assert plan.kernel(5) == "tensor_core"
    ntc = 0
    while True:
        try:
            plan.set_choice(5, ntc, 0)
        except _lib.FeiError:
            break
        if plan.kernel(5) == "sum_factorised":
            break
        ntc += 1
    assert ntc >= 2 and plan.kernel(5) == "sum_factorised"
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Ap, bp, sp, _ = plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], p=5)
        Ar, br, sr, _ = api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=5, precision="sf_fp32")
    s.synchronize()
    assert torch.equal(Ap, Ar) and torch.equal(bp, br)
    with pytest.raises(_lib.FeiError):
        plan.set_choice(5, ntc + 1, 0)


def test_plan_recapture_new_buffers_and_uniform():
    from paper_1310_1194_gb300 import api
    w, g, deg = _mixed(300)
    n = g["geom"].shape[0]
    layout = api.fei_plan_offsets(deg)
    plan = api.Plan(max_elem=n, precision="tc_f16x3")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A1, b1, _, _ = plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout)
        A2, b2, st2, _ = plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout)
    s.synchronize()
    assert torch.equal(A1, A2) and torch.equal(b1, b2) and int(st2.abs().max()) == 0
    # a uniform-degree batch through the same plan (p = 4, 37 elements)
    w4 = inputs.workload("p4", n_max=37)
    g4 = {k: torch.from_numpy(np.ascontiguousarray(w4[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    with torch.cuda.stream(s):
        A4, b4, st4, _ = plan.execute(g4["geom"], g4["K"], g4["b"], g4["c"], g4["f"], p=4)
    s.synchronize()
    Ao, bo, sto, _ = oracle.integrate(w4["geom"], w4["K"], w4["b"], w4["c"], w4["f"], p=4)
    Ah = A4.double().cpu().numpy().reshape(37, -1)
    for e in range(37):
        assert _rel(Ah[e], Ao.reshape(37, -1)[e]) <= 1e-6


def test_plan_rejects_oversized_batch():
    from paper_1310_1194_gb300 import api, _lib
    w, g, deg = _mixed(64)
    layout = api.fei_plan_offsets(deg)
    plan = api.Plan(max_elem=32, precision="fp32")
    with pytest.raises(_lib.FeiError) as ei:
        plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, layout=layout)
    assert ei.value.status == _lib.FEI_ERR_INVALID_ARG


def test_plan_tuning_cache_round_trip(tmp_path):
    """Choices saved by one plan and loaded into another give the same
    kernel shapes and the same results; a cache for another precision is
    not applied."""
    from paper_1310_1194_gb300 import api, _lib
    w, g, deg = _mixed(500)
    n = g["geom"].shape[0]
    layout = api.fei_plan_offsets(deg)
    args = (g["geom"], g["K"], g["b"], g["c"], g["f"])
    tuned = api.Plan(max_elem=n, precision="tc_f16x3")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tuned.tune(*args, degree=deg, layout=layout)
        A1, b1, _, _ = tuned.execute(*args, degree=deg, layout=layout)
    s.synchronize()
    path = str(tmp_path / "plan_cache.json")
    tuned.save_choices(path)
    loaded = api.Plan(max_elem=n, precision="tc_f16x3")
    assert loaded.load_choices(path)
    with torch.cuda.stream(s):
        A2, b2, st2, _ = loaded.execute(*args, degree=deg, layout=layout)
    s.synchronize()
    for p in range(1, 8):
        assert tuned.choice(p)[:2] == loaded.choice(p)[:2]
    assert torch.equal(A1, A2) and torch.equal(b1, b2) and int(st2.abs().max()) == 0
    other = api.Plan(max_elem=n, precision="fp32")
    before = [other.choice(p) for p in range(1, 8)]
    assert not other.load_choices(path)
    assert [other.choice(p) for p in range(1, 8)] == before
    with pytest.raises(_lib.FeiError):
        loaded.set_choice(4, 10 ** 6, 0)
    # tune() with a cache file applies the stored choices instead of timing,
    # and a plan of another precision adds its own entry
    third = api.Plan(max_elem=n, precision="tc_f16x3")
    with torch.cuda.stream(s):
        A3, b3, _, _ = third.tune(*args, degree=deg, layout=layout, cache=path)
        other.tune(*args, degree=deg, layout=layout, cache=path)
    s.synchronize()
    for p in range(1, 8):
        assert third.choice(p)[:2] == tuned.choice(p)[:2]
    assert torch.equal(A3, A1) and torch.equal(b3, b1)
    import json
    with open(path) as fh:
        assert len(json.load(fh)) == 2
