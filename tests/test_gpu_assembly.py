"""Assembly (Sec. 2) on the GPU against the assembly oracle: colour-by-colour
assembly of given element matrices, and integration fused with assembly,
for uniform and mixed degrees and per-point coefficients."""
import numpy as np
import pytest
import torch

import oracle
from oracle import assembly as oas
from paper_1310_1194_gb300 import inputs

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


def setup(api, name, n, shared="vertex"):
    w = inputs.workload(name, n_max=n)
    l2g, nd = inputs.dof_map(w, shared=shared)
    mixed = w["p"] is None
    asm = api.Assembly(l2g, nd, p=w["p"], degree=w["degree"] if mixed else None)
    return w, l2g, nd, asm


def oracle_system(w, l2g, nd):
    p = w["p"]
    A, b, st, _ = oracle.integrate(w["geom"], w["K"], w["b"], w["c"], w["f"], p=p,
                                   degree=None if p is not None else w["degree"], per_qp=w["per_qp"])
    return A, b, st, oas.assemble(A, b, l2g, nd, w["degree"])


def csr_close(rp, ci, v, orp, oci, ov, rtol):
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    scale = np.linalg.norm(ov)
    assert np.linalg.norm(v - ov) <= rtol * scale, np.linalg.norm(v - ov) / scale


@pytest.mark.parametrize("name,n", [("pr1", 400), ("mixed", 150), ("p4", 40)])
def test_assemble_given_element_matrices_fp64(api, name, n):
    """The oracle's element matrices assembled by the GPU, against the oracle's
    assembly of the same matrices (only the order of the sums differs)."""
    w, l2g, nd, asm = setup(api, name, n)
    A, b, _, (orp, oci, ov, orhs) = oracle_system(w, l2g, nd)
    values, rhs = asm.assemble(dev(A), dev(b), precision="fp64")
    torch.cuda.synchronize()
    rp, ci, colour = asm.pattern()
    csr_close(rp, ci, values.cpu().numpy(), orp, oci, ov, 1e-15)
    assert np.linalg.norm(rhs.cpu().numpy() - orhs) <= 1e-15 * np.linalg.norm(orhs)
    assert asm.n_colours == colour.max() + 1


def test_assemble_fp32(api):
    w, l2g, nd, asm = setup(api, "mixed", 120)
    A, b, _, (orp, oci, ov, orhs) = oracle_system(w, l2g, nd)
    values, rhs = asm.assemble(dev(A, torch.float32), dev(b, torch.float32), precision="fp32")
    torch.cuda.synchronize()
    rp, ci, _ = asm.pattern()
    csr_close(rp, ci, values.double().cpu().numpy(), orp, oci, ov, 1e-6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("tc_f16x3", 1e-6)])
@pytest.mark.parametrize("name,n", [("pr1", 300), ("mixed", 150), ("p4", 60)])
def test_integrate_assemble_against_the_oracle(api, precision, tol, name, n):
    w, l2g, nd, asm = setup(api, name, n)
    _, _, ost, (orp, oci, ov, orhs) = oracle_system(w, l2g, nd)
    deg = dev(w["degree"], torch.int32) if w["p"] is None else None
    values, rhs, st = asm.integrate_assemble(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                             precision=precision, degree=deg)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ost)
    rp, ci, _ = asm.pattern()
    csr_close(rp, ci, values.double().cpu().numpy(), orp, oci, ov, tol)
    assert np.linalg.norm(rhs.double().cpu().numpy() - orhs) <= tol * np.linalg.norm(orhs)


@pytest.mark.parametrize("precision", ["fp64", "tc_f16x3"])
def test_fused_equals_integrate_then_assemble(api, precision):
    """Chunked integration through the scratch gives the same element
    matrices as fei_integrate, so both assemblies agree to the last bit."""
    w, l2g, nd, asm = setup(api, "mixed", 400)
    deg = dev(w["degree"], torch.int32)
    g = [dev(w[k]) for k in ("geom", "K", "b", "c", "f")]
    A, b, st, _ = api.fei_integrate(*g, degree=deg, precision=precision)
    v1, r1 = asm.assemble(A, b, precision=precision)
    v2, r2, st2 = asm.integrate_assemble(*g, precision=precision, degree=deg)
    torch.cuda.synchronize()
    assert torch.equal(st, st2)
    assert torch.equal(v1, v2) and torch.equal(r1, r2)


def test_per_point_coefficients_fused(api):
    w, l2g, nd, asm = setup(api, "diff", 24)
    _, _, ost, (orp, oci, ov, orhs) = oracle_system(w, l2g, nd)
    values, rhs, st = asm.integrate_assemble(dev(w["geom"]), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                             precision="tc_f16x3", per_qp=True)
    torch.cuda.synchronize()
    rp, ci, _ = asm.pattern()
    csr_close(rp, ci, values.double().cpu().numpy(), orp, oci, ov, 1e-6)


def test_flagged_element_adds_nothing(api):
    """An inverted prism is flagged and its (zero) matrix adds nothing."""
    w, l2g, nd, asm = setup(api, "pr1", 50)
    w = dict(w)
    geom = w["geom"].copy()
    geom[7] = geom[7][[0, 2, 1, 3, 5, 4]]  # mirror element 7: det J < 0
    w["geom"] = geom
    _, _, ost, (orp, oci, ov, orhs) = oracle_system(w, l2g, nd)
    assert ost[7] != 0
    values, rhs, st = asm.integrate_assemble(dev(geom), dev(w["K"]), dev(w["b"]), dev(w["c"]), dev(w["f"]),
                                             precision="fp64")
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ost)
    rp, ci, _ = asm.pattern()
    csr_close(rp, ci, values.cpu().numpy(), orp, oci, ov, 1e-12)


def test_private_numbering_is_block_diagonal(api):
    w, l2g, nd, asm = setup(api, "mixed", 100, shared="none")
    assert asm.n_colours == 1
    deg = dev(w["degree"], torch.int32)
    g = [dev(w[k]) for k in ("geom", "K", "b", "c", "f")]
    A, b, st, _ = api.fei_integrate(*g, degree=deg, precision="fp64")
    values, rhs, _ = asm.integrate_assemble(*g, precision="fp64", degree=deg)
    torch.cuda.synchronize()
    assert torch.equal(values, A) and torch.equal(rhs, b)


def test_refused_arguments(api):
    from paper_1310_1194_gb300._lib import FeiError
    w, l2g, nd, asm = setup(api, "pr1", 20)
    g = [dev(w[k]) for k in ("geom", "K", "b", "c", "f")]
    with pytest.raises(FeiError, match="elements"):
        asm.integrate_assemble(g[0][:10], g[1][:10], g[2][:10], g[3][:10], g[4][:10], precision="fp64")
    host = api.Assembly(l2g, nd, p=1, host_only=True)
    with pytest.raises(FeiError, match="host-only"):
        host.assemble(dev(np.zeros(20 * 36)), dev(np.zeros(20 * 6)), precision="fp64")
