"""FP64 CPU oracle for prism element integration -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it: the oracle is ``fei_oracle.c`` (plain C, FP64,
Algorithm 1's loop order: element -> point -> i -> j -> k) compiled here with
gcc into ``oracle/_build/libfei_oracle.so`` and driven through ctypes.

Each function names the passage of the paper it follows:

* ``gauss_legendre``   -- Gaussian quadrature (Sec. 2, the accuracy rule
  "products of shape functions integrated exactly"); Newton on P_n.
* ``quadrature``       -- Duffy-collapsed Gauss-Legendre, (p+1)^3 points on the
  reference prism (Sec. 2; the paper names no rule, so the point count is a
  reading: exact for products of shape functions on affine prisms).
* ``basis``            -- prism shape functions: complete triangle basis times
  1D functions along the vertical direction (Table 1 and its text).
* ``integrate``        -- Eq. (2) generalised to
  int grad v.K grad u + v b.grad u + c u v  and  int f v, Algorithm 1.
* ``integrate_backward`` -- the reverse pass of ``integrate`` (hand-derived
  adjoint, FP64); derivative formulas are in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fei_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfei_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = 1
ERR_INVALID_DEGREE = 2
ERR_NEGATIVE_JACOBIAN = 3
ERR_NONFINITE = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so x86
    and aarch64 produce the same bits)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    compile_source(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    """Load a compiled oracle and declare its C signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lp = ctypes.POINTER(ctypes.c_int64)
    lib.fo_nsh.argtypes = [ctypes.c_int]
    lib.fo_nq.argtypes = [ctypes.c_int]
    lib.fo_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
    lib.fo_quadrature.argtypes = [ctypes.c_int, dp]
    lib.fo_basis.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, dp, dp]
    lib.fo_tabulate.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.fo_integrate.argtypes = [
        ctypes.c_int64, dp, ip, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
        lp, lp, lp, dp, dp, ip, ctypes.c_int]
    lib.fo_integrate_backward.argtypes = [
        ctypes.c_int64, dp, ip, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
        lp, lp, lp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
    return lib


def compile_source(src: str, out_path: str) -> str:
    """Compile an oracle C source (used by the mutation tests to build
    deliberately broken copies outside the package)."""
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fno-fast-math",
           "-ffp-contract=off", "-fPIC", "-shared", "-o", out_path, src,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    return out_path


_override = None


def use_library(path: str | None):
    """Point the module-level functions at another compiled oracle (None
    restores the default build)."""
    global _lib, _override
    with _lock:
        _override = path
        _lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(_override or build())
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def nsh(p: int) -> int:
    """Number of prism shape functions, (p+1)^2 (p+2)/2 (Table 1)."""
    return (p + 1) * (p + 1) * (p + 2) // 2


def nq(p: int) -> int:
    """Number of quadrature points of the Duffy rule, (p+1)^3."""
    return (p + 1) ** 3


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    rc = _load().fo_gauss_legendre(n, _ptr(x), _ptr(w))
    if rc:
        raise ValueError(f"gauss_legendre failed: {rc}")
    return x, w


def quadrature(p: int) -> np.ndarray:
    """[nq, 4] array of (xi1, xi2, zeta, w)."""
    pts = np.zeros((nq(p), 4))
    rc = _load().fo_quadrature(p, _ptr(pts))
    if rc:
        raise ValueError(f"quadrature failed: {rc}")
    return pts


def basis(p: int, xyz) -> tuple[np.ndarray, np.ndarray]:
    """Shape functions at reference points xyz [n, 3]: phi [n, nsh] and
    reference gradients dphi [n, nsh, 3]."""
    xyz = np.ascontiguousarray(np.atleast_2d(xyz), dtype=np.float64)
    n, s = xyz.shape[0], nsh(p)
    phi = np.zeros((n, s))
    dphi = np.zeros((n, s, 3))
    lib = _load()
    for k in range(n):
        rc = lib.fo_basis(p, float(xyz[k, 0]), float(xyz[k, 1]), float(xyz[k, 2]),
                          _ptr(phi[k]), _ptr(dphi[k]))
        if rc:
            raise ValueError(f"basis failed: {rc}")
    return phi, dphi


def _batch_arrays(geom, K, b, c, f, p, degree, per_qp, offsets):
    geom = np.ascontiguousarray(geom, dtype=np.float64).reshape(-1, 6, 3)
    n = geom.shape[0]
    K = np.ascontiguousarray(K, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    deg = None
    if degree is not None:
        deg = np.ascontiguousarray(degree, dtype=np.int32).reshape(n)
        degs = deg.astype(np.int64)
    else:
        if p is None:
            raise ValueError("give p or degree")
        degs = np.full(n, int(p), dtype=np.int64)
    if offsets is None:
        offsets = layout(degs)
    A_off, b_off, q_off = (np.ascontiguousarray(o, dtype=np.int64) for o in offsets)
    return geom, n, K, b, c, f, deg, A_off, b_off, q_off


def layout(degrees) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Contiguous output/coefficient offsets [n+1] for a degree list:
    A_e at A_off[e] (N_sh^2 scalars), b_e at b_off[e], per-point records at
    q_off[e]."""
    degs = np.asarray(degrees, dtype=np.int64)
    s = (degs + 1) * (degs + 1) * (degs + 2) // 2
    A_off = np.zeros(len(degs) + 1, dtype=np.int64)
    b_off = np.zeros(len(degs) + 1, dtype=np.int64)
    q_off = np.zeros(len(degs) + 1, dtype=np.int64)
    np.cumsum(s * s, out=A_off[1:])
    np.cumsum(s, out=b_off[1:])
    np.cumsum((degs + 1) ** 3, out=q_off[1:])
    return A_off, b_off, q_off


def integrate(geom, K, b, c, f, p=None, degree=None, per_qp=False, offsets=None,
              nthreads=0):
    """Element matrices and load vectors in FP64.

    Returns (A, bvec, status, offsets): A and bvec are flat arrays laid out by
    ``offsets`` = (A_off, b_off, q_off)."""
    geom, n, K, b, c, f, deg, A_off, b_off, q_off = _batch_arrays(
        geom, K, b, c, f, p, degree, per_qp, offsets)
    A = np.zeros(int(A_off[-1]))
    bv = np.zeros(int(b_off[-1]))
    st = np.zeros(n, dtype=np.int32)
    rc = _load().fo_integrate(
        n, _ptr(geom), _ptr(deg, ctypes.c_int32), int(p or 0), int(bool(per_qp)),
        _ptr(K), _ptr(b), _ptr(c), _ptr(f),
        _ptr(A_off, ctypes.c_int64), _ptr(b_off, ctypes.c_int64),
        _ptr(q_off, ctypes.c_int64), _ptr(A), _ptr(bv),
        _ptr(st, ctypes.c_int32), int(nthreads))
    if rc:
        raise ValueError(f"fo_integrate failed with status {rc}")
    return A, bv, st, (A_off, b_off, q_off)


def integrate_backward(geom, K, b, c, f, gA, gb, p=None, degree=None, per_qp=False,
                       offsets=None, nthreads=0):
    """Gradients of L = <gA, A> + <gb, b> w.r.t. geometry and coefficients.

    Returns (g_geom [n,6,3], gK, gb_coef, gc, gf) in the input layouts."""
    geom, n, K, b, c, f, deg, A_off, b_off, q_off = _batch_arrays(
        geom, K, b, c, f, p, degree, per_qp, offsets)
    gA = np.ascontiguousarray(gA, dtype=np.float64).reshape(-1)
    gb = np.ascontiguousarray(gb, dtype=np.float64).reshape(-1)
    g_geom = np.zeros((n, 6, 3))
    gK = np.zeros_like(K)
    gbc = np.zeros_like(b)
    gc = np.zeros_like(c)
    gf = np.zeros_like(f)
    rc = _load().fo_integrate_backward(
        n, _ptr(geom), _ptr(deg, ctypes.c_int32), int(p or 0), int(bool(per_qp)),
        _ptr(K), _ptr(b), _ptr(c), _ptr(f),
        _ptr(A_off, ctypes.c_int64), _ptr(b_off, ctypes.c_int64),
        _ptr(q_off, ctypes.c_int64), _ptr(gA), _ptr(gb), _ptr(g_geom),
        _ptr(gK), _ptr(gbc), _ptr(gc), _ptr(gf), int(nthreads))
    if rc:
        raise ValueError(f"fo_integrate_backward failed with status {rc}")
    return g_geom, gK, gbc, gc, gf


def split(flat, offsets_1d, sizes):
    """Split a flat output into per-element arrays (test helper)."""
    return [flat[int(offsets_1d[e]):int(offsets_1d[e]) + int(sizes[e])]
            for e in range(len(sizes))]
