"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative Frobenius norm per element, max over the batch; load
vectors by the 2-norm): FP64 path 1e-12, FP32 path 1e-5, split-precision
tensor-core path 1e-6, sum-factorised FP32 path 1e-5, gradients 1e-6 (FP32
contraction) / 1e-10 (FP64).
"""
import numpy as np
import pytest

import oracle
from paper_1310_1194_gb300 import inputs
from parity_util import assert_grads_close, worst_conditioned

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tc_f16x3": 1e-6, "tc_3xtf32": 1e-6, "sf_fp32": 1e-5}
# Gradients: element by element (relative Frobenius of the 18 vertex
# gradients, and of an element's per-point coefficient gradients) at the
# bars above, and record by record (one element's vertex gradients, one row
# of K, b, c or f) against max(the record's norm, the RMS of its group: the
# element's points, or the batch for per-element records).  FP64 at the
# element bar.  FP32 forms the per-point sums over the N_sh^2 random
# cotangents (and v_q = G_q u) in FP32: such a sum keeps about 1e-7 of the
# size of its terms, and a record that cancels to its group's RMS keeps
# that error relative to it (1.3e-6 measured at p = 5); 1e-5 bounds this
# with margin and still fails any record that is wrong (an index or sign
# mistake is an O(1) error).
TOL_GRAD_REC = {"fp64": 1e-10, "fp32": 1e-5, "tc_f16x3": 1e-5}
# elements per degree: several thread blocks / tiles and a ragged tail
N_PER_P = {1: 517, 2: 133, 3: 45, 4: 21, 5: 9, 6: 5, 7: 3}


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_1194_gb300 import api as a
    return a


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def per_elem_err(flat_gpu, flat_ref, offsets, sizes):
    errs = []
    for e in range(len(sizes)):
        o, s = int(offsets[e]), int(sizes[e])
        a, r = flat_gpu[o:o + s], flat_ref[o:o + s]
        nr = np.linalg.norm(r)
        errs.append(np.linalg.norm(a - r) / nr if nr > 0 else np.linalg.norm(a))
    return np.array(errs)


def run_gpu(api, w, p=None, degree=None, precision="fp64", per_qp=False):
    g = dev(w["geom"])
    A, bv, st, lay = api.fei_integrate(g, dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                       p=p, degree=None if degree is None else dev(degree),
                                       per_qp=per_qp, precision=precision)
    torch.cuda.synchronize()
    return A.double().cpu().numpy(), bv.double().cpu().numpy(), st.cpu().numpy()


def compare(api, w, p, precision, per_qp=False, degree=None):
    A, bv, st = run_gpu(api, w, p=p, degree=degree, precision=precision, per_qp=per_qp)
    Ao, bo, so, (Aoff, boff, _) = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"],
                                                  p=p, degree=degree, per_qp=per_qp)
    assert np.array_equal(st, so), (st[st != so][:5], so[st != so][:5])
    degs = np.full(len(w["geom"]), p) if degree is None else np.asarray(degree)
    s = (degs + 1) ** 2 * (degs + 2) // 2
    ea = per_elem_err(A, Ao, Aoff, s * s)
    eb = per_elem_err(bv, bo, boff, s)
    return ea, eb


def workload_for(p, n):
    return inputs.workload("p7", n_max=n) if p >= 6 else inputs.workload("pr1", n_max=n)


@pytest.mark.parametrize("p", range(1, 8))
def test_reference_tables_match_oracle(api, p):
    ref = api.fei_reference_create(p)
    pts, G = ref.table()
    pts_o = oracle.quadrature(p)
    assert np.max(np.abs(pts.numpy() - pts_o)) < 1e-15
    phi, dphi = oracle.basis(p, pts_o[:, :3])
    Go = np.concatenate([phi[:, None, :], dphi.transpose(0, 2, 1)], axis=1)
    scale = np.max(np.abs(Go))
    assert np.max(np.abs(G.numpy() - Go)) < 1e-13 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
@pytest.mark.parametrize("p", range(1, 8))
def test_forward_uniform_degree(api, p, precision):
    w = workload_for(p, N_PER_P[p])
    ea, eb = compare(api, w, p, precision)
    assert ea.max() < TOL[precision], (p, precision, ea.max())
    assert eb.max() < TOL[precision], (p, precision, eb.max())


def test_pr1_full_fp64(api):
    """PR1: 4096 prisms, p = 1, FP64 -- the whole batch."""
    w = inputs.workload("pr1")
    ea, eb = compare(api, w, 1, "fp64")
    assert ea.max() < 1e-12 and eb.max() < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
def test_mixed_degree_batch(api, precision):
    w = inputs.workload("mixed", n_max=240)
    ea, eb = compare(api, w, None, precision, degree=w["degree"])
    assert ea.max() < TOL[precision] and eb.max() < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
def test_per_point_coefficients(api, precision):
    w = inputs.workload("diff", n_max=6)
    ea, eb = compare(api, w, 5, precision, per_qp=True)
    assert ea.max() < TOL[precision] and eb.max() < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3", "tc_3xtf32", "sf_fp32"])
@pytest.mark.parametrize("p", [1, 4, 7])
def test_status_flags_and_zero_outputs(api, p, precision):
    w = workload_for(p, 7)
    geom = w["geom"].copy()
    geom[2] = geom[2][[0, 2, 1, 3, 5, 4]]  # mirrored: det J < 0
    c = w["c"].copy()
    c[4] = np.nan
    geom[5, 3, 1] = np.inf
    w2 = dict(w, geom=geom, c=c)
    A, bv, st = run_gpu(api, w2, p=p, precision=precision)
    s = api.nsh(p)
    assert list(st) == [0, 0, 3, 0, 4, 4, 0]
    for e in (2, 4, 5):
        assert np.all(A[e * s * s:(e + 1) * s * s] == 0) and np.all(bv[e * s:(e + 1) * s] == 0)
    ea, eb = compare(api, w2, p, precision)
    assert ea.max() < TOL[precision]


def test_custom_offsets_leave_gaps_untouched(api):
    """Caller-provided offsets with gaps between elements."""
    w = inputs.workload("pr1", n_max=5)
    p, s = 2, api.nsh(2)
    Aoff = np.arange(6, dtype=np.int64) * (s * s + 7)
    boff = np.arange(6, dtype=np.int64) * (s + 3)
    qoff = np.arange(6, dtype=np.int64) * api.nq(p)
    lay = api.Layout(dev(Aoff), dev(boff), dev(qoff), int(Aoff[-1]), int(boff[-1]), int(qoff[-1]))
    A = torch.full((lay.A_total,), 7.0, dtype=torch.float64, device="cuda")
    bv = torch.full((lay.b_total,), 7.0, dtype=torch.float64, device="cuda")
    st = torch.empty(5, dtype=torch.int32, device="cuda")
    deg = np.full(5, p, dtype=np.int32)
    api.fei_integrate(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                      degree=dev(deg), precision="fp64", layout=lay, out=(A, bv, st))
    A = A.cpu().numpy()
    Ao, bo, _, _ = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], p=p)
    for e in range(5):
        a = A[Aoff[e]:Aoff[e] + s * s]
        assert np.linalg.norm(a - Ao[e * s * s:(e + 1) * s * s]) < 1e-12 * np.linalg.norm(a)
        assert np.all(A[Aoff[e] + s * s:Aoff[e + 1]] == 7.0)


def test_empty_batch(api):
    z = torch.zeros((0, 6, 3), dtype=torch.float64, device="cuda")
    zK = torch.zeros((0, 3, 3), dtype=torch.float64, device="cuda")
    zb = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    zc = torch.zeros((0,), dtype=torch.float64, device="cuda")
    A, bv, st, _ = api.fei_integrate(z, zK, zb, zc, zc, p=3, precision="fp32")
    assert A.numel() == 0 and st.numel() == 0


def test_invalid_degree_reported(api):
    w = inputs.workload("pr1", n_max=4)
    with pytest.raises(api._lib.FeiError) as ei:
        api.fei_integrate(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]), p=9)
    assert ei.value.status == 2


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-6), ("tc_f16x3", 1e-6)])
@pytest.mark.parametrize("p,per_qp", [(1, False), (2, False), (3, False), (4, False), (5, True), (6, False),
                                     (7, False)])
def test_backward_matches_oracle_adjoint(api, p, per_qp, precision, tol):
    """The general adjoint against the oracle's, element by element and record
    by record.  tc_f16x3 forms dL/dDt on the tensor cores at p = 3..5 and
    runs the FP32 adjoint at the other degrees."""
    w = inputs.workload("diff", n_max=3) if per_qp else inputs.workload("p7", n_max=4)
    n = len(w["geom"])
    s = api.nsh(p)
    rng = np.random.default_rng(p)
    gA = rng.standard_normal(n * s * s)
    gb = rng.standard_normal(n * s)
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = api.fei_integrate_backward(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                     dev(gA, dt), dev(gb, dt), p=p, per_qp=per_qp, precision=precision)
    torch.cuda.synchronize()
    if precision != "fp64":  # the oracle sees the same rounded cotangents
        gA = gA.astype(np.float32).astype(np.float64)
        gb = gb.astype(np.float32).astype(np.float64)
    ref = oracle.integrate_backward(w["geom"], w["K"], w["b"], w["c"], w["f"], gA, gb, p=p, per_qp=per_qp)
    got = [t.cpu().numpy() for t in out]
    errs = assert_grads_close(got, ref, n, per_qp, np.full(n, api.nq(p)), tol, TOL_GRAD_REC[precision],
                              where=f"p={p} {precision}")
    print(f"adjoint p={p} {precision}:", {k: (float(v[0].max()) if len(v[0]) else None, float(v[1].max()))
                                            for k, v in errs.items()})


def test_autograd_matches_central_differences(api):
    """integrate() as a torch.autograd.Function: dL/dX and dL/dK of
    L = sum_e u_e^T A_e u_e - u_e^T b_e against central differences
    (h = 1e-6) of the FP64 GPU forward."""
    p, n = 3, 5
    w = inputs.workload("p7", n_max=n)
    s = api.nsh(p)
    u = torch.from_numpy(np.random.default_rng(7).standard_normal(n * s)).cuda()

    def loss(geom, K):
        A, bv, st = api.integrate(geom, K, dev(w["b"]), dev(w["c"]), dev(w["f"]), p=p, precision="fp64")
        Ae = A.view(n, s, s)
        ue = u.view(n, s)
        return (torch.einsum("ei,eij,ej->", ue, Ae, ue) - (ue * bv.view(n, s)).sum())

    geom = dev(w["geom"]).clone().requires_grad_(True)
    K = dev(w["K"]).clone().requires_grad_(True)
    L = loss(geom, K)
    L.backward()
    h = 1e-6
    for (t, idx) in [(geom, (0, 1, 2)), (geom, (3, 4, 0)), (geom, (4, 0, 1)), (K, (2, 0, 1)), (K, (1, 2, 2))]:
        base = (geom.detach(), K.detach())
        plus = [x.clone() for x in base]
        minus = [x.clone() for x in base]
        k = 0 if t is geom else 1
        plus[k][idx] += h
        minus[k][idx] -= h
        fd = (loss(*plus).item() - loss(*minus).item()) / (2 * h)
        got = t.grad[idx].item()
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (idx, got, fd)


@pytest.mark.parametrize("precision", ["tc_f16x3", "auto"])
def test_autograd_split_precision_uses_the_tensor_core_adjoint(api, precision):
    """integrate() with a split-precision forward at p = 4: its backward runs
    the tensor-core adjoint (gA from torch's autograd, a general cotangent,
    not u u^T), and the gradients of a loss with general weights on A and b
    match the FP64 autograd gradients element by element within the FP32
    bar."""
    p, n = 4, 40
    w = inputs.workload("p7", n_max=n)
    s = api.nsh(p)
    rng = np.random.default_rng(11)
    WA = torch.from_numpy(rng.standard_normal((n, s, s))).cuda()
    Wb = torch.from_numpy(rng.standard_normal((n, s))).cuda()

    def grads(prec):
        geom = dev(w["geom"]).clone().requires_grad_(True)
        K = dev(w["K"]).clone().requires_grad_(True)
        A, bv, st = api.integrate(geom, K, dev(w["b"]), dev(w["c"]), dev(w["f"]), p=p, precision=prec)
        L = (A.double().view(n, s, s) * WA).sum() + (bv.double().view(n, s) * Wb).sum()
        L.backward()
        return geom.grad.cpu().numpy(), K.grad.cpu().numpy()

    g64, k64 = grads("fp64")
    g, k = grads(precision)
    eg = np.linalg.norm((g - g64).reshape(n, -1), axis=1) / np.linalg.norm(g64.reshape(n, -1), axis=1)
    ek = np.linalg.norm((k - k64).reshape(n, -1), axis=1) / np.linalg.norm(k64.reshape(n, -1), axis=1)
    assert eg.max() < 1e-5 and ek.max() < 1e-5, (eg.max(), ek.max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
@pytest.mark.parametrize("p,per_qp", [(1, False), (4, False), (5, True), (7, False)])
def test_quadratic_adjoint_matches_oracle(api, p, per_qp, precision, tol):
    """fei_integrate_backward_quadratic equals the general adjoint of the
    oracle with gA_e = u_e u_e^T and gb_e = -u_e."""
    w = inputs.workload("diff", n_max=3) if per_qp else inputs.workload("p7", n_max=4)
    n = len(w["geom"])
    s = api.nsh(p)
    u = np.random.default_rng(10 + p).standard_normal(n * s)
    out = api.fei_integrate_backward_quadratic(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                               dev(u), p=p, per_qp=per_qp, precision=precision)
    torch.cuda.synchronize()
    ue = u.reshape(n, s)
    gA = np.einsum("ei,ej->eij", ue, ue).reshape(-1)
    ref = oracle.integrate_backward(w["geom"], w["K"], w["b"], w["c"], w["f"], gA, -u, p=p, per_qp=per_qp)
    got = [t.cpu().numpy() for t in out]
    errs = assert_grads_close(got, ref, n, per_qp, np.full(n, api.nq(p)), tol, TOL_GRAD_REC[precision],
                              where=f"quadratic p={p} {precision}")
    print(f"quadratic adjoint p={p} {precision}:",
          {k: (float(v[0].max()) if len(v[0]) else None, float(v[1].max())) for k, v in errs.items()})


def test_quadratic_adjoint_mixed_degrees(api):
    w = inputs.workload("mixed", n_max=60)
    deg = dev(w["degree"], torch.int32)
    layout = api.fei_plan_offsets(deg)
    u = np.random.default_rng(5).standard_normal(layout.b_total)
    out = api.fei_integrate_backward_quadratic(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                               dev(u), degree=deg, layout=layout, precision="fp64")
    torch.cuda.synchronize()
    boff = layout.b_offset.cpu().numpy()
    gA = np.concatenate([np.outer(u[boff[e]:boff[e + 1]], u[boff[e]:boff[e + 1]]).reshape(-1)
                         for e in range(len(w["geom"]))])
    ref = oracle.integrate_backward(w["geom"], w["K"], w["b"], w["c"], w["f"], gA, -u, degree=w["degree"])
    got = [t.cpu().numpy() for t in out]
    assert_grads_close(got, ref, len(w["geom"]), False, None, 1e-10, TOL_GRAD_REC["fp64"], where="mixed fp64")


def test_status_summary(api):
    st = torch.tensor([0, 3, 0, 4, 3, 0, 7, 0], dtype=torch.int32, device="cuda")
    assert api.fei_status_summary(st) == (4, 4)
    st = torch.tensor([0, 3, 0, 0], dtype=torch.int32, device="cuda")
    assert api.fei_status_summary(st) == (3, 1)
    st = torch.zeros(100000, dtype=torch.int32, device="cuda")
    assert api.fei_status_summary(st) == (0, 0)
    st[77777] = 6
    assert api.fei_status_summary(st) == (6, 1)


def test_sync_status_reads_the_summary_on_the_host(api):
    """fei_sync_status after a forward with flagged elements: the worst code
    and the count of fei_status_summary, as host values, once the stream has
    finished the forward."""
    w = workload_for(4, 7)
    geom = w["geom"].copy()
    geom[2] = geom[2][[0, 2, 1, 3, 5, 4]]  # det J < 0
    c = w["c"].copy()
    c[4] = np.nan
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        A, bv, st, _ = api.fei_integrate(dev(geom), dev(w["K"]), dev(w["b"]), dev(c), dev(w["f"]), p=4,
                                         precision="tc_f16x3")
        assert api.fei_sync_status(st) == (4, 2)
    assert list(st.cpu().numpy()) == [0, 0, 3, 0, 4, 0, 0]
    assert api.fei_sync_status(torch.zeros(0, dtype=torch.int32, device="cuda")) == (0, 0)
    z = torch.zeros(300000, dtype=torch.int32, device="cuda")
    z[123456] = 3
    assert api.fei_sync_status(z) == (3, 1)


@pytest.mark.parametrize("p", [3, 4, 5])
def test_tc_output_not_16_byte_aligned(api, p):
    """A_out starting 4 bytes past an aligned address (and b_out likewise):
    the tensor-core path must fall back from its bulk stores and still match
    the oracle element by element."""
    w = inputs.workload("p4", n_max=41)
    n = len(w["geom"])
    s = api.nsh(p)
    Abuf = torch.zeros(n * s * s + 1, dtype=torch.float32, device="cuda")
    bbuf = torch.zeros(n * s + 1, dtype=torch.float32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    A, bv = Abuf[1:], bbuf[1:]
    api.fei_integrate(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]), p=p,
                      precision="tc_f16x3", out=(A, bv, st))
    torch.cuda.synchronize()
    assert float(Abuf[0]) == 0.0 and float(bbuf[0]) == 0.0
    Ao, bo, so, _ = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], p=p)
    Ah = A.double().cpu().numpy().reshape(n, -1)
    Aor = Ao.reshape(n, -1)
    for e in range(n):
        assert np.linalg.norm(Ah[e] - Aor[e]) <= 1e-6 * np.linalg.norm(Aor[e]), e


def test_plan_per_point_coefficients_mixed(api):
    """A plan over a mixed batch with per-point coefficient records."""
    w = inputs.workload("mixed", n_max=90)
    deg = dev(w["degree"], torch.int32)
    layout = api.fei_plan_offsets(deg)
    q = (w["degree"].astype(np.int64) + 1) ** 3
    rng = np.random.default_rng(3)
    m = int(q.sum())
    K = np.broadcast_to(np.eye(3), (m, 3, 3)).copy() * rng.uniform(0.5, 2.0, size=(m, 1, 1))
    b = rng.uniform(-1, 1, size=(m, 3))
    c = rng.uniform(0, 1, size=m)
    f = rng.uniform(-1, 1, size=m)
    plan = api.Plan(max_elem=len(w["geom"]), precision="tc_f16x3")
    s_ = torch.cuda.Stream()
    with torch.cuda.stream(s_):
        A, bv, st, _ = plan.execute(dev(w["geom"]), dev(K), dev(b), dev(c), dev(f), degree=deg, per_qp=True,
                                    layout=layout)
    s_.synchronize()
    Ao, bo, so, _ = oracle.integrate(w["geom"], K, b, c, f, degree=w["degree"], per_qp=True)
    assert int(st.abs().max()) == 0 and int(np.abs(so).max()) == 0
    Ah = A.double().cpu().numpy()
    Aoff = layout.A_offset.cpu().numpy()
    for e in range(len(w["geom"])):
        sl = slice(int(Aoff[e]), int(Aoff[e + 1]))
        assert np.linalg.norm(Ah[sl] - Ao[sl]) <= 1e-6 * np.linalg.norm(Ao[sl]), (e, int(w["degree"][e]))


def test_coefficient_arrays_of_the_wrong_length_are_refused(api):
    """Per-point records sized for p = 5 given with p = 6: refused before any
    launch (the kernels cannot see the arrays' lengths)."""
    w = inputs.workload("diff", n_max=4)
    g = {k: dev(w[k]) for k in ("geom", "K", "b", "c", "f")}
    with pytest.raises(ValueError, match="per quadrature point"):
        api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=6, per_qp=True, precision="fp64")
    with pytest.raises(ValueError, match="per element"):
        api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=5, per_qp=False, precision="fp64")


@pytest.mark.parametrize("p", [4, 5])
def test_tc_operand_scale_covers_every_point(api, p):
    """Per-point diffusion 10^4 times larger at the last quadrature point of
    every element: each element's fp16 operand scale must come from the bound
    of all its points (a scale that missed that point would overflow fp16)."""
    n = 9
    w = inputs.workload("pr1", n_max=n)
    q = (p + 1) ** 3
    K = np.broadcast_to(np.eye(3), (n, q, 3, 3)).copy()
    K[:, -1] *= 1e4
    K = K.reshape(n * q, 3, 3)
    b = np.full((n * q, 3), 0.1)
    c = np.full(n * q, 0.5)
    f = np.ones(n * q)
    A, bv, st, _ = api.fei_integrate(dev(w["geom"]), dev(K), dev(b), dev(c), dev(f), p=p, per_qp=True,
                                     precision="tc_f16x3")
    torch.cuda.synchronize()
    Ao, bo, so, _ = oracle.integrate(w["geom"], K, b, c, f, p=p, per_qp=True)
    assert int(st.abs().max()) == 0 and int(np.abs(so).max()) == 0
    Ah = A.double().cpu().numpy().reshape(n, -1)
    assert np.isfinite(Ah).all()
    Aor = Ao.reshape(n, -1)
    for e in range(n):
        assert np.linalg.norm(Ah[e] - Aor[e]) <= 1e-6 * np.linalg.norm(Aor[e]), e


def test_tc_wait_timeout_reports_status_and_context_survives(api):
    """Fault injection: with a 1 us limit on the tensor-core forward's
    pipeline waits, blocks give up, flag their remaining elements
    FEI_ERR_TIMEOUT and return without any fault; elements of tiles that
    finished keep exact results, and the next launch with the default limit
    is whole and correct."""
    from paper_1310_1194_gb300 import _lib
    w = inputs.workload("p4", n_max=3000)
    g = [dev(w[k]) for k in ("geom", "K", "b", "c", "f")]
    _lib.check(_lib.lib.fei_debug_set_wait_limit(1000), "fei_debug_set_wait_limit")
    try:
        A, bv, st, _ = api.fei_integrate(*g, p=4, precision="tc_f16x3")
        torch.cuda.synchronize()
    finally:
        _lib.check(_lib.lib.fei_debug_set_wait_limit(0), "fei_debug_set_wait_limit")
    stc = st.cpu().numpy()
    assert (stc == _lib.FEI_ERR_TIMEOUT).sum() > 0
    assert set(np.unique(stc).tolist()) <= {0, _lib.FEI_ERR_TIMEOUT}
    A2, b2, st2, _ = api.fei_integrate(*g, p=4, precision="tc_f16x3")
    torch.cuda.synchronize()
    assert int(st2.abs().max()) == 0
    s = api.nsh(4)
    done = np.flatnonzero(stc == 0)
    if len(done):
        Ad = A.view(-1, s * s)[torch.from_numpy(done).cuda()]
        assert torch.equal(Ad, A2.view(-1, s * s)[torch.from_numpy(done).cuda()])
    idx = np.array([0, 1500, 2999])
    Ao, bo, so, _ = oracle.integrate(w["geom"][idx], w["K"][idx], w["b"][idx], w["c"][idx], w["f"][idx], p=4)
    Ah = A2.view(-1, s * s)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    for j in range(len(idx)):
        ao = Ao[j * s * s:(j + 1) * s * s]
        assert np.linalg.norm(Ah[j] - ao) <= 1e-6 * np.linalg.norm(ao)


@pytest.mark.parametrize("bprec", ["fp64", "fp32"])
def test_p5_per_point_gradients_match_central_differences(api, bprec):
    """The differentiation workload's configuration (p = 5, coefficients per
    quadrature point): dL/dX and dL/d(K, b, c, f) of L = sum_e u_e^T A_e u_e
    - u_e^T b_e from the library's adjoints (the quadratic-loss adjoint and
    the general one through autograd) against central differences of the
    FP64 GPU forward, per-point values held fixed."""
    p, n = 5, 3
    w = inputs.workload("diff", n_max=n)
    s, q = api.nsh(p), api.nq(p)
    u = np.random.default_rng(21).standard_normal(n * s)
    ud = dev(u)
    g = {k: dev(w[k]) for k in ("geom", "K", "b", "c", "f")}

    def outputs(x):
        A, bv, st, _ = api.fei_integrate(x["geom"], x["K"], x["b"], x["c"], x["f"], p=p, per_qp=True,
                                         precision="fp64")
        assert not st.any()
        return A.view(n, s, s), bv.view(n, s)

    def loss_difference(plus, minus):
        # L(plus) - L(minus) from the differences of the outputs: entries the
        # step does not touch cancel exactly, so the rounding of L itself
        # (about 1e-16 |L|) does not enter
        (Ap, bp), (Am, bm) = outputs(plus), outputs(minus)
        ue = ud.view(n, s)
        return float((torch.einsum("ei,eij,ej->", ue, Ap - Am, ue) - (ue * (bp - bm)).sum()).item())

    quad = api.fei_integrate_backward_quadratic(g["geom"], g["K"], g["b"], g["c"], g["f"], ud, p=p, per_qp=True,
                                                precision=bprec)
    geom = g["geom"].clone().requires_grad_(True)
    Kt = g["K"].clone().requires_grad_(True)
    ct = g["c"].clone().requires_grad_(True)
    A, bv, st = api.integrate(geom, Kt, g["b"], ct, g["f"], p=p, per_qp=True, precision=bprec)
    L = torch.einsum("ei,eij,ej->", ud.view(n, s).to(A.dtype), A.view(n, s, s), ud.view(n, s).to(A.dtype)) - \
        (ud.view(n, s).to(bv.dtype) * bv.view(n, s)).sum()
    L.backward()
    tol = 1e-6 if bprec == "fp64" else 1e-5
    checks = [("geom", (0, 1, 2)), ("geom", (2, 4, 0)), ("geom", (1, 3, 1)), ("K", (17, 0, 1)), ("K", (q + 40, 2, 2)),
              ("b", (2 * q + 7, 1)), ("c", (q + 100,)), ("f", (2 * q + 211,))]
    names = ("geom", "K", "b", "c", "f")
    for name, idx in checks:
        # A_e and b_e are linear in K, b, c and f (the weak form of Sec. 2),
        # so the central difference is exact there whatever the step: a
        # unit one keeps the rounding of the outputs small against the step
        h = 1e-6 if name == "geom" else 1.0
        plus = {k: v.clone() for k, v in g.items()}
        minus = {k: v.clone() for k, v in g.items()}
        plus[name][idx] += h
        minus[name][idx] -= h
        fd = loss_difference(plus, minus) / (2 * h)
        got_q = float(quad[names.index(name)][idx])
        scale = float(quad[names.index(name)].abs().max())
        assert abs(got_q - fd) <= tol * max(abs(fd), 1e-2 * scale), ("quadratic", name, idx, got_q, fd)
        auto = {"geom": geom, "K": Kt, "c": ct}.get(name)
        if auto is not None:
            got_a = float(auto.grad[idx])
            assert abs(got_a - fd) <= tol * max(abs(fd), 1e-2 * scale), ("autograd", name, idx, got_a, fd)


@pytest.mark.parametrize("upper", [False, True])
def test_p1_small_and_large_batches_give_the_same_bits(api, upper):
    """At p = 1 the FP32 path runs eight lanes per element for small batches
    and one thread per element for large ones; both give the same bits (the
    host-memory entry cuts a batch into chunks of any size), and the oracle
    agrees with both."""
    w = inputs.workload("p1m", n_max=20000)
    if upper:
        K = np.asarray(w["K"]).reshape(-1, 3, 3)
        w = dict(w, K=np.ascontiguousarray((0.5 * (K + np.swapaxes(K, 1, 2))).reshape(w["K"].shape)),
                 b=np.zeros_like(w["b"]))
    big = api.fei_integrate(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]), p=1,
                            precision="fp32", upper=upper)
    m = 3001
    small = api.fei_integrate(dev(w["geom"][:m]), dev(w["K"][:m]), dev(w["b"][:m]), dev(w["c"][:m]),
                              dev(w["f"][:m]), p=1, precision="fp32", upper=upper)
    torch.cuda.synchronize()
    s = api.a_size(1, upper)
    Ab, bb, sb = (x.cpu().numpy() for x in big[:3])
    As, bs, ss = (x.cpu().numpy() for x in small[:3])
    assert not sb.any() and not ss.any()
    assert np.array_equal(As.view(np.uint8), Ab[:m * s].view(np.uint8))
    assert np.array_equal(bs.view(np.uint8), bb[:m * 6].view(np.uint8))
    idx = np.array([0, 1234, 3000])
    Ao, bo, so, _ = oracle.integrate(w["geom"][idx], w["K"][idx], w["b"][idx], w["c"][idx], w["f"][idx], p=1)
    full = As.reshape(m, s).astype(np.float64)
    if upper:
        full = api.unpack_upper(full, 1).reshape(m, 36)
    for k, e in enumerate(idx):
        ref = Ao[36 * k:36 * (k + 1)]
        assert np.linalg.norm(full[e] - ref) <= 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["tc_f16x3", "tc_3xtf32", "fp32"])
@pytest.mark.parametrize("p", [3, 4])
def test_far_and_tiny_coordinates(api, p, precision):
    """Element set-up of the tensor-core path on coordinates that stress
    it: elements moved 1e4 and 1e6 from the origin (vertex differences far
    below the coordinates), and elements with an edge of length 1e-20 along
    one axis (a vertex difference outside the range of the exact FP32 split,
    so the element takes the FP64 steps) mixed into one batch.  Parity
    with the oracle at the same bar as the plain workload."""
    w = workload_for(p, 24)
    geom = w["geom"].copy().reshape(24, 6, 3)
    geom[0:8] += np.array([1.0e4, -3.0e4, 2.0e4])
    geom[8:16] += np.array([-1.0e6, 0.0, 0.5e6])
    # vertices 0 and 3 (one vertical edge) share x and y, and vertex 3's y
    # moves by 1e-20: the difference X_3 - X_0 has a y component of 1e-20
    geom[16:24:2, 3, :2] = geom[16:24:2, 0, :2]
    geom[16:24:2, 3, 1] += 1e-20 if p == 3 else -1e-20
    w = dict(w, geom=np.ascontiguousarray(geom.reshape(w["geom"].shape)))
    ea, eb = compare(api, w, p, precision)
    assert ea.max() < TOL[precision], (p, precision, ea.max())
    assert eb.max() < TOL[precision], (p, precision, eb.max())


@pytest.mark.parametrize("p,per_qp", [(3, False), (4, False), (5, True)])
def test_tc_adjoint_blocks_and_chunks(api, monkeypatch, p, per_qp):
    """The tensor-core adjoint over more elements than thread blocks (each
    block's pipeline runs several elements: B buffers, A stages and
    accumulator buffers wrap) and over several launch chunks (the chain reads
    the scratch at an element offset), with cotangents whose rows differ by
    orders of magnitude (each gA row has its own split scale: over six
    orders, one scale per element would leave the small rows about 18 bits
    of fp16 hi + lo instead of 22)."""
    n = {3: 400, 4: 170, 5: 160}[p]
    w = inputs.workload("diff", n_max=n) if per_qp else inputs.workload("p7", n_max=n)
    n = len(w["geom"])
    s = api.nsh(p)
    rng = np.random.default_rng(100 + p)
    row_scale = 10.0 ** rng.integers(-3, 4, size=(n, s, 1))
    gA = (rng.standard_normal((n, s, s)) * row_scale).reshape(-1)
    gb = rng.standard_normal(n * s)
    monkeypatch.setenv("FEI_ADJOINT_CHUNK", "64")
    out = api.fei_integrate_backward(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                     dev(gA, torch.float32), dev(gb, torch.float32), p=p, per_qp=per_qp,
                                     precision="tc_f16x3")
    torch.cuda.synchronize()
    gA = gA.astype(np.float32).astype(np.float64)
    gb = gb.astype(np.float32).astype(np.float64)
    ref = oracle.integrate_backward(w["geom"], w["K"], w["b"], w["c"], w["f"], gA, gb, p=p, per_qp=per_qp)
    got = [t.cpu().numpy() for t in out]
    assert_grads_close(got, ref, n, per_qp, np.full(n, api.nq(p)), 1e-6, TOL_GRAD_REC["tc_f16x3"],
                       where=f"p={p} tc_f16x3, {n} elements in chunks of 64")
