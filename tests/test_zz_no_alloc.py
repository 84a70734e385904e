"""fei_integrate_noalloc against fei_integrate, through the C ABI (GPU).

fei_integrate_noalloc is for callers that cannot let the library allocate
device memory (stream capture, code that must not block the device, memory
owned by a pool): its degree-bucketing scratch is a fixed device array.
This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
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


def _batch(_lib, g, deg, lay):
    bt = _lib.fei_batch()
    bt.n_elem = g["geom"].shape[0]
    bt.geom = g["geom"].data_ptr()
    bt.degree = deg.data_ptr()
    bt.uniform_degree = 0
    bt.coef_mode = _lib.FEI_COEF_PER_ELEMENT
    bt.K, bt.b, bt.c, bt.f = (g[k].data_ptr() for k in ("K", "b", "c", "f"))
    bt.A_offset = lay.A_offset.data_ptr()
    bt.b_offset = lay.b_offset.data_ptr()
    bt.q_offset = lay.q_offset.data_ptr()
    return bt


@pytest.mark.parametrize("precision", ["fp32", "tc_f16x3"])
def test_noalloc_matches_fei_integrate_twice(env, precision):
    _lib, api = env
    lib = _lib.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    refs = [api.fei_reference_create(p) for p in range(1, 8)]
    rarr = (ctypes.c_void_p * 7)(*[r.handle.value for r in refs])
    prec = _lib.PRECISIONS[precision]
    for call, (n, offset) in enumerate(((700, 0), (523, 900))):  # two calls in a row, different batches
        w = inputs.workload("mixed", n_max=offset + n)
        g = {k: torch.from_numpy(np.ascontiguousarray(w[k][offset:])).cuda() for k in ("geom", "K", "b", "c", "f")}
        deg = torch.from_numpy(np.ascontiguousarray(w["degree"][offset:])).cuda()
        lay = api.fei_plan_offsets(deg)
        bt = _batch(_lib, g, deg, lay)
        outs = []
        for fn in (lib.fei_integrate, lib.fei_integrate_noalloc):
            A = torch.full((lay.A_total,), float("nan"), dtype=torch.float32, device="cuda")
            bv = torch.full((lay.b_total,), float("nan"), dtype=torch.float32, device="cuda")
            st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            rc = fn(rarr, 7, ctypes.byref(bt), prec, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(bv.data_ptr()),
                    ctypes.c_void_p(st.data_ptr()), stream)
            assert rc == 0, _lib.last_error()
            torch.cuda.synchronize()
            outs.append((A.double().cpu().numpy(), bv.double().cpu().numpy(), st.cpu().numpy()))
        (A0, b0, s0), (A1, b1, s1) = outs
        assert np.array_equal(s0, s1) and not s1.any()
        Ao = lay.A_offset.cpu().numpy()
        degs = w["degree"][offset:]
        sizes = ((degs + 1) ** 2 * (degs + 2) // 2) ** 2
        for e in range(n):
            a0 = A0[Ao[e]:Ao[e] + sizes[e]]
            a1 = A1[Ao[e]:Ao[e] + sizes[e]]
            assert np.linalg.norm(a1 - a0) <= 1e-6 * np.linalg.norm(a0), (call, e)
        assert np.allclose(b1, b0, rtol=1e-6, atol=0)


def test_noalloc_rejects_oversized_batch(env):
    _lib, api = env
    lib = _lib.lib
    bt = _lib.fei_batch()
    bt.n_elem = _lib.FEI_NOALLOC_MAX_ELEM + 1
    rc = lib.fei_integrate_noalloc(None, 0, ctypes.byref(bt), _lib.FEI_FP32, None, None, None, None)
    assert rc == _lib.FEI_ERR_INVALID_ARG
    assert "capacity" in _lib.last_error()
