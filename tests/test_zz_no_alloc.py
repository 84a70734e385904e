"""fei_integrate_noalloc against fei_integrate, through the C ABI (GPU).

fei_integrate_noalloc is for callers that cannot let the library allocate
device memory -- code that must never block the device (cudaMalloc can
synchronise it), or memory owned by a pool or budget: its degree-bucketing
scratch is a fixed device array.  After the bucketing it runs the same
kernels on the same elements as fei_integrate, so the outputs must agree
bit for bit.  This file is collected last so that a failure here comes
after every other test has run; it also passes on its own in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_1310_1194_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_1194_gb300 import _lib, api
    return _lib, api


def _batch(_lib, g, deg, lay, p=0):
    bt = _lib.fei_batch()
    bt.n_elem = g["geom"].shape[0]
    bt.geom = g["geom"].data_ptr()
    bt.degree = deg.data_ptr() if deg is not None else None
    bt.uniform_degree = p
    bt.coef_mode = _lib.FEI_COEF_PER_ELEMENT
    bt.K, bt.b, bt.c, bt.f = (g[k].data_ptr() for k in ("K", "b", "c", "f"))
    bt.A_offset = lay.A_offset.data_ptr() if lay.A_offset is not None else None
    bt.b_offset = lay.b_offset.data_ptr() if lay.b_offset is not None else None
    bt.q_offset = lay.q_offset.data_ptr() if lay.q_offset is not None else None
    return bt


def _both(_lib, refs, bt, prec, lay, n):
    """Runs fei_integrate, then fei_integrate_noalloc, on the same batch into
    NaN-filled outputs; returns both results as host arrays."""
    lib = _lib.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rarr = (ctypes.c_void_p * len(refs))(*[r.handle.value for r in refs])
    dt = torch.float64 if prec == _lib.FEI_FP64 else torch.float32
    outs = []
    for fn in (lib.fei_integrate, lib.fei_integrate_noalloc):
        A = torch.full((lay.A_total,), float("nan"), dtype=dt, device="cuda")
        bv = torch.full((lay.b_total,), float("nan"), dtype=dt, device="cuda")
        st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = fn(rarr, len(refs), ctypes.byref(bt), prec, ctypes.c_void_p(A.data_ptr()),
                ctypes.c_void_p(bv.data_ptr()), ctypes.c_void_p(st.data_ptr()), stream)
        assert rc == 0, _lib.last_error()
        torch.cuda.synchronize()
        outs.append((A.cpu().numpy(), bv.cpu().numpy(), st.cpu().numpy()))
    return outs


def _equal_bits(x, y):
    """Same values bit for bit, NaNs (untouched output) included."""
    return x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tc_f16x3"])
def test_noalloc_matches_fei_integrate_twice(env, precision):
    """Two calls in a row on different mixed-degree batches: each equals
    fei_integrate bit for bit (the second call starts from the array the
    first one left behind)."""
    _lib, api = env
    refs = [api.fei_reference_create(p) for p in range(1, 8)]
    prec = _lib.PRECISIONS[precision]
    for call, (n, offset) in enumerate(((700, 0), (523, 900))):
        w = inputs.workload("mixed", n_max=offset + n)
        g = {k: torch.from_numpy(np.ascontiguousarray(w[k][offset:])).cuda() for k in ("geom", "K", "b", "c", "f")}
        deg = torch.from_numpy(np.ascontiguousarray(w["degree"][offset:])).cuda()
        lay = api.fei_plan_offsets(deg)
        (A0, b0, s0), (A1, b1, s1) = _both(_lib, refs, _batch(_lib, g, deg, lay), prec, lay, n)
        assert np.array_equal(s0, s1) and not s1.any(), call
        assert not np.isnan(A1).any() and not np.isnan(b1).any(), call
        assert _equal_bits(A0, A1) and _equal_bits(b0, b1), call


def test_noalloc_partial_references_give_the_same_statuses(env):
    """References for degrees 2, 4 and 7 only: elements of the other degrees
    get FEI_ERR_INVALID_DEGREE and untouched outputs, exactly as with
    fei_integrate."""
    _lib, api = env
    refs = [api.fei_reference_create(p) for p in (2, 4, 7)]
    n = 400
    w = inputs.workload("mixed", n_max=n)
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    deg = torch.from_numpy(np.ascontiguousarray(w["degree"])).cuda()
    lay = api.fei_plan_offsets(deg)
    (A0, b0, s0), (A1, b1, s1) = _both(_lib, refs, _batch(_lib, g, deg, lay), _lib.FEI_TC_F16X3, lay, n)
    want = np.where(np.isin(w["degree"], (2, 4, 7)), 0, _lib.FEI_ERR_INVALID_DEGREE)
    assert np.array_equal(s1, want) and np.array_equal(s0, s1)
    assert _equal_bits(A0, A1) and _equal_bits(b0, b1)


def test_noalloc_uniform_degree_batch(env):
    """degree = NULL: a uniform batch needs no scratch and is fei_integrate's
    own call."""
    _lib, api = env
    p, n = 4, 300
    refs = [api.fei_reference_create(p)]
    w = inputs.workload("p4", n_max=n)
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).cuda() for k in ("geom", "K", "b", "c", "f")}
    lay = api.uniform_layout(n, p)
    (A0, b0, s0), (A1, b1, s1) = _both(_lib, refs, _batch(_lib, g, None, lay, p), _lib.FEI_TC_F16X3, lay, n)
    assert not s1.any() and np.array_equal(s0, s1)
    assert _equal_bits(A0, A1) and _equal_bits(b0, b1)


def test_noalloc_rejects_oversized_batch(env):
    _lib, api = env
    lib = _lib.lib
    bt = _lib.fei_batch()
    bt.n_elem = _lib.FEI_NOALLOC_MAX_ELEM + 1
    rc = lib.fei_integrate_noalloc(None, 0, ctypes.byref(bt), _lib.FEI_FP32, None, None, None, None)
    assert rc == _lib.FEI_ERR_INVALID_ARG
    assert "capacity" in _lib.last_error()
