"""Python binding with the C ABI's names (include/fei.h).

PyTorch provides device memory and the current CUDA stream; every step of
the integration runs in libfei's kernels.  All tensors are CUDA tensors on
the current device; inputs are FP64 and contiguous.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check, lib


def nsh(p: int) -> int:
    return (p + 1) * (p + 1) * (p + 2) // 2


def nq(p: int) -> int:
    return (p + 1) ** 3


def a_size(p: int, upper: bool = False) -> int:
    """Values of one A_e: N_sh^2, or N_sh (N_sh + 1) / 2 as its upper triangle."""
    s = nsh(p)
    return s * (s + 1) // 2 if upper else s * s


def unpack_upper(a_upper, p: int):
    """The full N_sh x N_sh matrices of elements stored as upper triangles
    (row i holds A[i][i..N_sh-1]): a_upper [..., N_sh (N_sh + 1) / 2] ->
    [..., N_sh, N_sh], mirrored across the diagonal (a torch tensor or a
    numpy array; no kernel)."""
    s = nsh(p)
    iu = np.triu_indices(s)
    if isinstance(a_upper, torch.Tensor):
        out = a_upper.new_zeros(a_upper.shape[:-1] + (s, s))
        r, c = torch.as_tensor(iu[0], device=a_upper.device), torch.as_tensor(iu[1], device=a_upper.device)
        out[..., r, c] = a_upper
        out[..., c, r] = a_upper
        return out
    a_upper = np.asarray(a_upper)
    out = np.zeros(a_upper.shape[:-1] + (s, s), dtype=a_upper.dtype)
    out[..., iu[0], iu[1]] = a_upper
    out[..., iu[1], iu[0]] = a_upper
    return out


class Reference:
    """Owning wrapper of a fei_reference_t (reference data of degree p)."""

    def __init__(self, p: int):
        h = ctypes.c_void_p()
        check(lib.fei_reference_create(int(p), ctypes.byref(h)), "fei_reference_create")
        self.handle = h
        self.p = int(p)
        self.nsh = nsh(p)
        self.nq = nq(p)
        self.device = torch.cuda.current_device()

    def table(self):
        """(pts [N_q, 4], G [N_q, 4, N_sh]) as FP64 host tensors."""
        pts = torch.zeros(self.nq, 4, dtype=torch.float64)
        G = torch.zeros(self.nq, 4, self.nsh, dtype=torch.float64)
        check(lib.fei_reference_copy_table(self.handle, pts.data_ptr(), G.data_ptr()),
              "fei_reference_copy_table")
        return pts, G

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fei_reference_destroy(h)
            self.handle = None


_ref_cache: dict[tuple[int, int], Reference] = {}


def fei_reference_create(p: int) -> Reference:
    """Reference data of degree p on the current device (cached per device)."""
    key = (torch.cuda.current_device(), int(p))
    r = _ref_cache.get(key)
    if r is None:
        r = Reference(p)
        _ref_cache[key] = r
    return r


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, name, dtype=torch.float64):
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


@dataclass
class Layout:
    """Output layout of a batch: per-element offsets (device int64 [n+1],
    or None for the contiguous uniform-degree layout) and total sizes."""
    A_offset: torch.Tensor | None
    b_offset: torch.Tensor | None
    q_offset: torch.Tensor | None
    A_total: int
    b_total: int
    q_total: int


def fei_plan_offsets(degree: torch.Tensor, upper: bool = False) -> Layout:
    """Contiguous offsets of a degree array (computed by a kernel); upper:
    for A_e stored as upper triangles."""
    degree = _need(degree, "degree", torch.int32)
    n = degree.numel()
    dev = degree.device
    Ao = torch.empty(n + 1, dtype=torch.int64, device=dev)
    bo = torch.empty(n + 1, dtype=torch.int64, device=dev)
    qo = torch.empty(n + 1, dtype=torch.int64, device=dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    fn = lib.fei_plan_offsets_upper if upper else lib.fei_plan_offsets
    check(fn(_ptr(degree), n, _ptr(Ao), _ptr(bo), _ptr(qo), _ptr(bad), _stream()), "fei_plan_offsets")
    tail = torch.stack([Ao[-1], bo[-1], qo[-1], bad[0].to(torch.int64)]).cpu().tolist()
    if tail[3]:
        raise ValueError(f"{tail[3]} elements have a degree outside 1..7")
    return Layout(Ao, bo, qo, int(tail[0]), int(tail[1]), int(tail[2]))


def fei_status_summary(status: torch.Tensor):
    """(worst status, number of flagged elements) of a status array, reduced
    on the device (one small copy back)."""
    status = _need(status, "status", torch.int32)
    out = torch.zeros(2, dtype=torch.int32, device=status.device)
    check(lib.fei_status_summary(_ptr(status), status.numel(), _ptr(out), _stream()), "fei_status_summary")
    worst, count = out.cpu().tolist()
    return int(worst), int(count)


def fei_sync_status(status: torch.Tensor):
    """(worst status, number of flagged elements) of a status array: the
    library reduces it on the current stream, waits for the stream and
    returns host values (fei_sync_status of the C ABI)."""
    status = _need(status, "status", torch.int32)
    worst, count = ctypes.c_int32(), ctypes.c_int64()
    check(lib.fei_sync_status(_ptr(status), status.numel(), ctypes.byref(worst), ctypes.byref(count), _stream()),
          "fei_sync_status")
    return int(worst.value), int(count.value)


def uniform_layout(n: int, p: int, upper: bool = False) -> Layout:
    s = nsh(p)
    return Layout(None, None, None, n * a_size(p, upper), n * s, n * nq(p))


def _batch(geom, K, b, c, f, degree, p, per_qp, layout, upper=False):
    n = geom.shape[0]
    bt = _lib.fei_batch()
    bt.n_elem = n
    bt.geom = geom.data_ptr()
    bt.degree = degree.data_ptr() if degree is not None else None
    bt.uniform_degree = int(p) if p is not None else 0
    bt.coef_mode = _lib.FEI_COEF_PER_POINT if per_qp else _lib.FEI_COEF_PER_ELEMENT
    bt.K = K.data_ptr()
    bt.b = b.data_ptr()
    bt.c = c.data_ptr()
    bt.f = f.data_ptr()
    bt.A_offset = layout.A_offset.data_ptr() if layout.A_offset is not None else None
    bt.b_offset = layout.b_offset.data_ptr() if layout.b_offset is not None else None
    bt.q_offset = layout.q_offset.data_ptr() if layout.q_offset is not None else None
    bt.a_layout = _lib.FEI_A_UPPER if upper else _lib.FEI_A_FULL
    return bt


def _refs_array(refs):
    arr = (ctypes.c_void_p * len(refs))(*[r.handle.value for r in refs])
    return arr


def _inputs(geom, K, b, c, f, degree, p, per_qp, layout, upper=False):
    geom = _need(geom, "geom")
    if geom.dim() != 3 or geom.shape[1:] != (6, 3):
        raise ValueError("geom must be [n, 6, 3]")
    for t, name in ((K, "K"), (b, "b"), (c, "c"), (f, "f")):
        _need(t, name)
    if degree is not None:
        _need(degree, "degree", torch.int32)
        if layout is None:
            layout = fei_plan_offsets(degree, upper)
    else:
        if p is None:
            raise ValueError("give p or degree")
        if layout is None:
            layout = uniform_layout(geom.shape[0], p, upper)
    # the kernels index the coefficient records by element (or by element
    # and point) without knowing the arrays' lengths, so a short array would
    # be read past its end: its size is checked here
    m = layout.q_total if per_qp else geom.shape[0]
    for t, name, width in ((K, "K", 9), (b, "b", 3), (c, "c", 1), (f, "f", 1)):
        if t.numel() != width * m:
            per = "quadrature point" if per_qp else "element"
            raise ValueError(f"{name} must hold {width} values per {per} ({width * m} in all), got {t.numel()}")
    return geom, layout


def fei_integrate(geom, K, b, c, f, p=None, degree=None, per_qp=False, precision="fp32",
                  refs=None, layout=None, out=None, upper=False):
    """Element matrices and load vectors (forward, Algorithm 1).

    Returns (A, b_vec, status, layout): A [A_total] and b_vec [b_total] in
    FP64 for precision "fp64" and FP32 otherwise, laid out by ``layout``;
    status int32 [n].  upper: each A_e as its upper triangle (a symmetric
    weak form: b = 0 and K symmetric; see unpack_upper)."""
    geom, layout = _inputs(geom, K, b, c, f, degree, p, per_qp, layout, upper)
    prec = _lib.PRECISIONS[precision]
    dtype = torch.float64 if prec == _lib.FEI_FP64 else torch.float32
    n = geom.shape[0]
    if refs is None:
        degs = [int(p)] if degree is None else list(range(1, 8))
        refs = [fei_reference_create(d) for d in degs]
    if out is None:
        A = torch.empty(layout.A_total, dtype=dtype, device=geom.device)
        bv = torch.empty(layout.b_total, dtype=dtype, device=geom.device)
        st = torch.empty(n, dtype=torch.int32, device=geom.device)
    else:
        A, bv, st = out
    bt = _batch(geom, K, b, c, f, degree, p, per_qp, layout, upper)
    check(lib.fei_integrate(_refs_array(refs), len(refs), ctypes.byref(bt), prec,
                            _ptr(A), _ptr(bv), _ptr(st), _stream()), "fei_integrate")
    return A, bv, st, layout


def fei_integrate_backward(geom, K, b, c, f, gA, gb, p=None, degree=None, per_qp=False,
                           precision="fp64", refs=None, layout=None):
    """Gradients of <gA, A> + <gb, b>: (g_geom, gK, gb_coef, gc, gf), FP64.

    precision: "fp64" (gA, gb FP64; all FP64), "fp32" (gA, gb FP32; the FP32
    adjoint), "tc_f16x3" or "auto" (gA, gb FP32; at a uniform degree 3..5
    dL/dDt is formed on the tensor cores, elsewhere the FP32 adjoint runs);
    other split precisions run the FP32 adjoint."""
    geom, layout = _inputs(geom, K, b, c, f, degree, p, per_qp, layout)
    prec = _lib.PRECISIONS[precision]
    dtype = torch.float64 if prec == _lib.FEI_FP64 else torch.float32
    _need(gA, "gA", dtype)
    _need(gb, "gb", dtype)
    if refs is None:
        degs = [int(p)] if degree is None else list(range(1, 8))
        refs = [fei_reference_create(d) for d in degs]
    g_geom = torch.empty_like(geom)
    gK = torch.empty_like(K)
    gbc = torch.empty_like(b)
    gc = torch.empty_like(c)
    gf = torch.empty_like(f)
    cg = _lib.fei_coef_grad(gK.data_ptr(), gbc.data_ptr(), gc.data_ptr(), gf.data_ptr())
    bt = _batch(geom, K, b, c, f, degree, p, per_qp, layout)
    check(lib.fei_integrate_backward(_refs_array(refs), len(refs), ctypes.byref(bt), prec,
                                     _ptr(gA), _ptr(gb), _ptr(g_geom), ctypes.byref(cg), _stream()),
          "fei_integrate_backward")
    return g_geom, gK, gbc, gc, gf


def fei_integrate_backward_quadratic(geom, K, b, c, f, u, p=None, degree=None, per_qp=False,
                                     precision="fp64", refs=None, layout=None):
    """Gradients of L = sum_e u_e^T A_e u_e - u_e^T b_e with respect to the
    geometry and the coefficients, (g_geom, gK, gb_coef, gc, gf) in FP64,
    without forming gA (u: FP64 [b_total] in the layout of b)."""
    geom, layout = _inputs(geom, K, b, c, f, degree, p, per_qp, layout)
    prec = _lib.PRECISIONS[precision]
    _need(u, "u")
    if refs is None:
        degs = [int(p)] if degree is None else list(range(1, 8))
        refs = [fei_reference_create(d) for d in degs]
    g_geom = torch.empty_like(geom)
    gK = torch.empty_like(K)
    gbc = torch.empty_like(b)
    gc = torch.empty_like(c)
    gf = torch.empty_like(f)
    cg = _lib.fei_coef_grad(gK.data_ptr(), gbc.data_ptr(), gc.data_ptr(), gf.data_ptr())
    bt = _batch(geom, K, b, c, f, degree, p, per_qp, layout)
    check(lib.fei_integrate_backward_quadratic(_refs_array(refs), len(refs), ctypes.byref(bt), prec, _ptr(u),
                                               _ptr(g_geom), ctypes.byref(cg), _stream()),
          "fei_integrate_backward_quadratic")
    return g_geom, gK, gbc, gc, gf


class Plan:
    """Owning wrapper of a fei_plan_t: a (mixed-degree) batch executed as one
    CUDA graph, with per-degree kernel shapes from the autotuner.

    ``execute`` takes the same arguments as :func:`fei_integrate` (outputs
    must be given with ``out`` for the graph to be replayed: a new output
    buffer means a new capture)."""

    def __init__(self, degrees=range(1, 8), max_elem: int = 0, precision: str = "tc_f16x3"):
        self.precision = precision
        self.refs = [fei_reference_create(d) for d in degrees]
        self.max_elem = int(max_elem)
        h = ctypes.c_void_p()
        check(lib.fei_plan_create(_refs_array(self.refs), len(self.refs), self.max_elem,
                                  _lib.PRECISIONS[precision], ctypes.byref(h)), "fei_plan_create")
        self.handle = h

    def _call(self, fn, name, geom, K, b, c, f, p, degree, per_qp, layout, out, upper=False):
        geom, layout = _inputs(geom, K, b, c, f, degree, p, per_qp, layout, upper)
        prec = _lib.PRECISIONS[self.precision]
        dtype = torch.float64 if prec == _lib.FEI_FP64 else torch.float32
        n = geom.shape[0]
        if out is None:
            A = torch.empty(layout.A_total, dtype=dtype, device=geom.device)
            bv = torch.empty(layout.b_total, dtype=dtype, device=geom.device)
            st = torch.empty(n, dtype=torch.int32, device=geom.device)
        else:
            A, bv, st = out
        bt = _batch(geom, K, b, c, f, degree, p, per_qp, layout, upper)
        check(fn(self.handle, ctypes.byref(bt), _ptr(A), _ptr(bv), _ptr(st), _stream()), name)
        return A, bv, st, layout

    def execute(self, geom, K, b, c, f, p=None, degree=None, per_qp=False, layout=None, out=None, upper=False):
        return self._call(lib.fei_plan_execute, "fei_plan_execute", geom, K, b, c, f, p, degree, per_qp,
                          layout, out, upper)

    def tune(self, geom, K, b, c, f, p=None, degree=None, per_qp=False, layout=None, out=None, cache=None):
        """Times the candidate kernel shapes of every degree on this batch
        and keeps the fastest.  With a cache file (``cache``, else the
        environment variable FEI_AUTOTUNE_CACHE) holding choices for this GPU
        model and precision, those are applied instead of timing; otherwise
        the tuned choices are added to it."""
        path = cache if cache is not None else os.environ.get("FEI_AUTOTUNE_CACHE")
        if path and os.path.exists(path) and self.load_choices(path):
            return self.execute(geom, K, b, c, f, p, degree, per_qp, layout, out)
        result = self._call(lib.fei_plan_tune, "fei_plan_tune", geom, K, b, c, f, p, degree, per_qp,
                            layout, out)
        if path:
            torch.cuda.current_stream().synchronize()
            self.save_choices(path)
        return result

    def choice(self, p: int):
        """(variant, grid cap in blocks, tuned ms) chosen for degree p."""
        v, g, t = ctypes.c_int(), ctypes.c_int64(), ctypes.c_float()
        check(lib.fei_plan_choice(self.handle, int(p), ctypes.byref(v), ctypes.byref(g), ctypes.byref(t)),
              "fei_plan_choice")
        return v.value, g.value, t.value

    def kernel(self, p: int) -> str:
        """The kernel the current choice runs for degree p: "cuda_core",
        "tensor_core" or "sum_factorised"."""
        k = ctypes.c_int32()
        check(lib.fei_plan_kernel(self.handle, int(p), ctypes.byref(k)), "fei_plan_kernel")
        return _lib.KERNELS[k.value]

    def set_choice(self, p: int, variant: int, grid_cap: int):
        check(lib.fei_plan_set_choice(self.handle, int(p), int(variant), int(grid_cap)), "fei_plan_set_choice")

    def _cache_key(self):
        return f"{torch.cuda.get_device_name()}|{self.precision}"

    def save_choices(self, path: str):
        """The tuning cache: this plan's per-degree choices, added to the
        JSON file under the key "<GPU model>|<precision>" (other keys kept)."""
        import json
        data = {}
        if os.path.exists(path):
            with open(path) as fh:
                data = json.load(fh)
        data[self._cache_key()] = {str(p): dict(zip(("variant", "grid_cap", "tuned_ms"), self.choice(p)))
                                   for p in range(1, 8)}
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(tmp, path)

    def load_choices(self, path: str) -> bool:
        """Applies the choices stored for this GPU model and precision;
        returns False (and changes nothing) if the file has none."""
        import json
        with open(path) as fh:
            data = json.load(fh)
        entry = data.get(self._cache_key())
        if entry is None:
            return False
        for p, c in entry.items():
            self.set_choice(int(p), c["variant"], c["grid_cap"])
        return True

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fei_plan_destroy(h)
            self.handle = None


def _host_f64(t, name, dtype=torch.float64):
    if t is None:
        raise ValueError(f"{name} is required")
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host {dtype} tensor")
    return t


class Pipeline:
    """Owning wrapper of a fei_pipeline_t: integration of a batch held in
    host memory, chunk by chunk through two device slots, the copies of one
    chunk overlapping the integration of the next (include/fei.h).

    ``integrate_host`` takes host tensors (page-locked ones let the copies
    overlap) and returns host tensors (A, b_vec, status) packed in element
    order, complete once the current stream has reached them."""

    def __init__(self, degrees=range(1, 8), precision: str = "tc_f16x3", slot_bytes: int = 0, refs=None):
        self.precision = precision
        self.refs = list(refs) if refs is not None else [fei_reference_create(d) for d in degrees]
        h = ctypes.c_void_p()
        check(lib.fei_pipeline_create(_refs_array(self.refs), len(self.refs), _lib.PRECISIONS[precision],
                                      int(slot_bytes), ctypes.byref(h)), "fei_pipeline_create")
        self.handle = h
        sb, me = ctypes.c_int64(), ctypes.c_int64()
        check(lib.fei_pipeline_info(h, ctypes.byref(sb), ctypes.byref(me)), "fei_pipeline_info")
        self.slot_bytes, self.max_elem = sb.value, me.value
        self.n_chunks = 0

    def totals(self, n, p=None, degree=None, per_qp=False, upper=False):
        """(A_total, b_total, record count) of the packed layout (A_e as
        upper triangles with upper=True)."""
        if degree is None:
            s, q = (p + 1) ** 2 * (p + 2) // 2, (p + 1) ** 3
            return n * (s * (s + 1) // 2 if upper else s * s), n * s, n * q if per_qp else n
        d = degree.numpy().astype(np.int64)
        ok = (d >= 1) & (d <= 7)
        s = np.where(ok, (d + 1) ** 2 * (d + 2) // 2, 0)
        q = np.where(ok, (d + 1) ** 3, 0)
        a = s * (s + 1) // 2 if upper else s * s
        return int(a.sum()), int(s.sum()), int(q.sum()) if per_qp else n

    def integrate_host(self, geom, K, b, c, f, p=None, degree=None, per_qp=False, out=None, upper=False):
        geom = _host_f64(geom, "geom")
        if geom.dim() != 3 or geom.shape[1:] != (6, 3):
            raise ValueError("geom must be [n, 6, 3]")
        if degree is not None:
            _host_f64(degree, "degree", torch.int32)
        elif p is None:
            raise ValueError("give p or degree")
        n = geom.shape[0]
        A_total, b_total, m = self.totals(n, p, degree, per_qp, upper)
        for t, name, width in ((K, "K", 9), (b, "b", 3), (c, "c", 1), (f, "f", 1)):
            _host_f64(t, name)
            if t.numel() != width * m:
                per = "quadrature point" if per_qp else "element"
                raise ValueError(f"{name} must hold {width} values per {per} ({width * m} in all), got {t.numel()}")
        dtype = torch.float64 if self.precision == "fp64" else torch.float32
        if out is None:
            A = torch.empty(A_total, dtype=dtype, pin_memory=True)
            bv = torch.empty(b_total, dtype=dtype, pin_memory=True)
            st = torch.empty(n, dtype=torch.int32, pin_memory=True)
        else:
            A, bv, st = out
            for t, name, size, dt in ((A, "A", A_total, dtype), (bv, "b_vec", b_total, dtype),
                                      (st, "status", n, torch.int32)):
                _host_f64(t, name, dt)
                if t.numel() != size:
                    raise ValueError(f"{name} must hold {size} values, got {t.numel()}")
        bt = _lib.fei_batch()
        bt.n_elem = n
        bt.geom = geom.data_ptr()
        bt.degree = degree.data_ptr() if degree is not None else None
        bt.uniform_degree = int(p) if p is not None else 0
        bt.coef_mode = _lib.FEI_COEF_PER_POINT if per_qp else _lib.FEI_COEF_PER_ELEMENT
        bt.K, bt.b, bt.c, bt.f = K.data_ptr(), b.data_ptr(), c.data_ptr(), f.data_ptr()
        bt.a_layout = _lib.FEI_A_UPPER if upper else _lib.FEI_A_FULL
        nc = ctypes.c_int64()
        check(lib.fei_integrate_host(self.handle, ctypes.byref(bt), _ptr(A), _ptr(bv), _ptr(st),
                                     ctypes.byref(nc), _stream()), "fei_integrate_host")
        self.n_chunks = nc.value
        return A, bv, st

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fei_pipeline_destroy(h)
            self.handle = None


class Assembly:
    """Assembly of element matrices into a global CSR matrix (Sec. 2).

    ``l2g``: host int64 array, element e's N_sh(p_e) global numbers at the
    element's load-vector offset; ``n_dof``: number of global functions.
    The pattern, a colouring of the elements (elements that share a global
    function get different colours) and the scatter map are built on the
    host; ``assemble`` then adds the element matrices colour by colour
    without atomics, and ``integrate_assemble`` integrates and assembles
    chunk by chunk through an L2-sized scratch.  ``host_only`` builds the
    pattern and colouring without touching a GPU."""

    def __init__(self, l2g, n_dof, p=None, degree=None, host_only=False):
        l2g = np.ascontiguousarray(l2g, dtype=np.int64)
        if degree is not None:
            self.degree = np.ascontiguousarray(degree, dtype=np.int32)
            n = len(self.degree)
            deg_ptr = self.degree.ctypes.data
        else:
            if p is None:
                raise ValueError("give p or degree")
            self.degree = None
            n = len(l2g) // nsh(p)
            deg_ptr = None
        self.p, self.n_elem, self.host_only = p, n, host_only
        self._l2g = l2g
        h = ctypes.c_void_p()
        check(lib.fei_assembly_create(n, deg_ptr, int(p or 0), l2g.ctypes.data, int(n_dof),
                                      1 if host_only else 0, ctypes.byref(h)), "fei_assembly_create")
        self.handle = h
        self.n_dof, self.nnz, self.n_colours, self.n_chunks = self.info()

    def info(self):
        """(n_dof, nnz, colours, chunks of the fused path)."""
        a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        check(lib.fei_assembly_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                    ctypes.byref(d)), "fei_assembly_info")
        return a.value, b.value, c.value, d.value

    def pattern(self):
        """Host copies: row_ptr int64 [n_dof + 1], col_idx int32 [nnz],
        colour int32 [n_elem]."""
        rp = np.empty(self.n_dof + 1, dtype=np.int64)
        ci = np.empty(max(self.nnz, 1), dtype=np.int32)
        co = np.empty(self.n_elem, dtype=np.int32)
        check(lib.fei_assembly_pattern(self.handle, rp.ctypes.data, ci.ctypes.data, co.ctypes.data),
              "fei_assembly_pattern")
        return rp, ci[: self.nnz], co

    def _outputs(self, precision, device, out):
        dtype = torch.float64 if precision == "fp64" else torch.float32
        if out is not None:
            return out
        return (torch.empty(self.nnz, dtype=dtype, device=device),
                torch.empty(self.n_dof, dtype=dtype, device=device))

    def assemble(self, A, bvec, precision="fp32", out=None):
        """values [nnz], rhs [n_dof] from A, b in fei_integrate's layout."""
        dtype = torch.float64 if precision == "fp64" else torch.float32
        for t, name in ((A, "A"), (bvec, "b")):
            if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
        values, rhs = self._outputs(precision, A.device, out)
        check(lib.fei_assemble(self.handle, _lib.PRECISIONS[precision], _ptr(A), _ptr(bvec), _ptr(values),
                               _ptr(rhs), _stream()), "fei_assemble")
        return values, rhs

    def integrate_assemble(self, geom, K, b, c, f, precision="fp32", per_qp=False, degree=None, refs=None,
                           out=None):
        """Fused integration and assembly; returns (values, rhs, status).
        ``degree``: device int32 tensor of the handle's degrees (a mixed
        batch), else the handle's uniform degree is used."""
        p = None if degree is not None else self.p
        geom, layout = _inputs(geom, K, b, c, f, degree, p, per_qp, None)
        if refs is None:
            degs = [int(p)] if degree is None else sorted(set(int(x) for x in self.degree))
            refs = [fei_reference_create(d) for d in degs]
        values, rhs = self._outputs(precision, geom.device, None if out is None else out[:2])
        st = torch.empty(geom.shape[0], dtype=torch.int32, device=geom.device) if out is None else out[2]
        bt = _batch(geom, K, b, c, f, degree, p, per_qp, layout)
        check(lib.fei_integrate_assemble(self.handle, _refs_array(refs), len(refs), ctypes.byref(bt),
                                         _lib.PRECISIONS[precision], _ptr(values), _ptr(rhs), _ptr(st),
                                         _stream()), "fei_integrate_assemble")
        return values, rhs, st

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fei_assembly_destroy(h)
            self.handle = None


class _IntegrateFn(torch.autograd.Function):
    """A, b = integrate(geom, K, b, c, f) with the library's adjoint kernel
    as the backward; the Jacobians are recomputed in the backward."""

    @staticmethod
    def forward(ctx, geom, K, bc, c, f, p, degree, per_qp, precision, layout):
        A, bv, st, layout = fei_integrate(geom, K, bc, c, f, p=p, degree=degree, per_qp=per_qp,
                                          precision=precision, layout=layout)
        ctx.save_for_backward(geom, K, bc, c, f)
        ctx.cfg = (p, degree, per_qp, precision, layout)
        ctx.mark_non_differentiable(st)
        return A, bv, st

    @staticmethod
    def backward(ctx, gA, gb, _gst):
        geom, K, bc, c, f = ctx.saved_tensors
        p, degree, per_qp, precision, layout = ctx.cfg
        # the tensor-core adjoint where the forward ran the split fp16 path
        # (the library runs it at a uniform degree 3..5, else the FP32 one)
        bprec = "fp64" if precision == "fp64" else "tc_f16x3" if precision in ("tc_f16x3", "auto") else "fp32"
        dt = torch.float64 if bprec == "fp64" else torch.float32
        gA = torch.zeros(layout.A_total, dtype=dt, device=geom.device) if gA is None else gA.to(dt).contiguous()
        gb = torch.zeros(layout.b_total, dtype=dt, device=geom.device) if gb is None else gb.to(dt).contiguous()
        g = fei_integrate_backward(geom, K, bc, c, f, gA, gb, p=p, degree=degree, per_qp=per_qp,
                                   precision=bprec, layout=layout)
        return (*g, None, None, None, None, None)


def integrate(geom, K, b, c, f, p=None, degree=None, per_qp=False, precision="fp32", layout=None):
    """Differentiable element integration: returns (A, b_vec, status)."""
    if degree is not None and layout is None:
        layout = fei_plan_offsets(degree)
    if degree is None and layout is None:
        layout = uniform_layout(geom.shape[0], p)
    return _IntegrateFn.apply(geom, K, b, c, f, p, degree, per_qp, precision, layout)
