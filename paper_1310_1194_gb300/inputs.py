"""Seeded synthetic inputs for prism element integration.

This module only makes inputs: jittered prism meshes, coefficient sets and
degree lists.  It holds none of the integration arithmetic (no quadrature, no
basis, no element matrices), and both the CUDA path and the CPU oracle take
their inputs from it.

Workloads (all seeded, numpy PCG64):

* ``pr1``   -- 16x16x8 unit-cube grid, each hex split into 2 prisms (4096),
  vertex jitter +-10% of h, p = 1, per-element coefficients.
* ``p4``    -- 50x50x20 grid (100 000 prisms), +-10% h, p = 4.
* ``mixed`` -- 50x50x40 grid (200 000 prisms), +-10% h, degree drawn per
  element from {1..7} with probabilities {.25,.2,.15,.15,.1,.1,.05}.
* ``diff``  -- 25x20x20 grid (20 000 prisms), +-10% h, p = 5, coefficients
  varying per quadrature slot (smooth sin/cos fields of position).
* ``p7``    -- 32x32x16 grid (32 768 prisms), +-25% h with every element
  certified valid (positive Jacobian determinant), p = 7.
* ``p1m``   -- 100x100x50 grid (1 000 000 prisms), +-10% h, p = 1: the
  PR1 recipe at a size where the store-bound low-degree path is measurable.
* ``p4sym`` -- the ``p4`` batch with b = 0: a symmetric weak form (K is
  symmetric), whose element matrices can be stored as upper triangles.

Coefficients per element: K = Q diag(lam) Q^T with Q from the QR factor of a
3x3 standard normal matrix (sign-fixed) and lam ~ U[0.5, 2]; b ~ U[-1, 1]^3;
c ~ U[0, 1]; f ~ U[-1, 1].
"""
from __future__ import annotations

import numpy as np

MIXED_PROBS = (0.25, 0.2, 0.15, 0.15, 0.1, 0.1, 0.05)

WORKLOADS = {
    "pr1": dict(grid=(16, 16, 8), jitter=0.10, seed=1, p=1),
    "p4": dict(grid=(50, 50, 20), jitter=0.10, seed=2, p=4),
    "mixed": dict(grid=(50, 50, 40), jitter=0.10, seed=3, p=None),
    "diff": dict(grid=(25, 20, 20), jitter=0.10, seed=4, p=5),
    "p7": dict(grid=(32, 32, 16), jitter=0.25, seed=5, p=7),
    "p1m": dict(grid=(100, 100, 50), jitter=0.10, seed=6, p=1),
    "p4sym": dict(grid=(50, 50, 20), jitter=0.10, seed=2, p=4, symmetric=True),
}


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def _prism_vertices(nx, ny, nz):
    """Vertex ids [n_prism, 6] of the structured grid: every hex column quad
    (i,j) is split along its (i,j)-(i+1,j+1) diagonal into two counter-
    clockwise triangles, extruded from layer k to k+1 (bottom 0,1,2, top
    3,4,5 above them)."""
    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ii = ii.transpose(2, 1, 0).reshape(-1)  # k slowest, then j, then i
    jj = jj.transpose(2, 1, 0).reshape(-1)
    kk = kk.transpose(2, 1, 0).reshape(-1)
    v00 = vid(ii, jj, kk)
    v10 = vid(ii + 1, jj, kk)
    v11 = vid(ii + 1, jj + 1, kk)
    v01 = vid(ii, jj + 1, kk)
    up = (nx + 1) * (ny + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.stack([t1, t2], axis=1).reshape(-1, 3)
    return np.concatenate([tri, tri + up], axis=1)


def _element_valid(geom: np.ndarray) -> np.ndarray:
    """Validity certificate of bilinear prisms [n, 6, 3].

    The map's Jacobian determinant is affine in the triangle coordinates at
    fixed height and quadratic in the height, so it is positive on the whole
    element iff, over each of the three vertical edges, the quadratic in
    height is positive on [-1, 1].  Returns a bool mask."""
    P, Q = geom[:, :3], geom[:, 3:]
    ok = np.ones(geom.shape[0], dtype=bool)

    def edge_det(t):
        s0, s1 = 0.5 * (1 - t), 0.5 * (1 + t)
        e1 = s0 * (P[:, 1] - P[:, 0]) + s1 * (Q[:, 1] - Q[:, 0])
        e2 = s0 * (P[:, 2] - P[:, 0]) + s1 * (Q[:, 2] - Q[:, 0])
        return np.cross(e1, e2)

    n_m, n_0, n_p = edge_det(-1.0), edge_det(0.0), edge_det(1.0)
    for a in range(3):
        v = 0.5 * (Q[:, a] - P[:, a])
        gm = np.einsum("ij,ij->i", n_m, v)
        g0 = np.einsum("ij,ij->i", n_0, v)
        gp = np.einsum("ij,ij->i", n_p, v)
        # g(t) = g0 + t (gp - gm)/2 + t^2 ((gp + gm)/2 - g0)
        b1 = 0.5 * (gp - gm)
        b2 = 0.5 * (gp + gm) - g0
        ok &= (gm > 0) & (gp > 0) & (g0 > 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            t_star = np.where(b2 > 0, -b1 / (2 * b2), 0.0)
        inside = (b2 > 0) & (t_star > -1) & (t_star < 1)
        gmin = g0 + t_star * b1 + t_star * t_star * b2
        ok &= ~inside | (gmin > 0)
    return ok


def prism_mesh(nx: int, ny: int, nz: int, jitter: float, seed: int,
               max_redraws: int = 100) -> np.ndarray:
    """Jittered prism mesh of the unit cube: geometry [2 nx ny nz, 6, 3] FP64.

    Every vertex (boundary ones too) moves by U[-jitter h, jitter h] per axis
    (h = 1/n per axis), so neighbouring prisms stay conforming.  Elements that
    fail the validity certificate get their vertices redrawn from the same
    random stream (at most ``max_redraws`` rounds), and any left invalid get
    zero jitter on their vertices; the result is deterministic per seed."""
    rng = _rng(seed, 0)
    gx = np.linspace(0.0, 1.0, nx + 1)
    gy = np.linspace(0.0, 1.0, ny + 1)
    gz = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    base = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    jit = rng.uniform(-jitter, jitter, size=base.shape) * h
    pv = _prism_vertices(nx, ny, nz)
    for _ in range(max_redraws):
        geom = (base + jit)[pv]
        bad = ~_element_valid(geom)
        if not bad.any():
            return geom
        verts = np.unique(pv[bad].reshape(-1))
        jit[verts] = rng.uniform(-jitter, jitter, size=(len(verts), 3)) * h
    while True:
        geom = (base + jit)[pv]
        bad = ~_element_valid(geom)
        if not bad.any():
            return geom
        jit[np.unique(pv[bad].reshape(-1))] = 0.0


def coefficients(n: int, seed: int) -> dict:
    """Per-element coefficient set: K [n,3,3] SPD, b [n,3], c [n], f [n]."""
    rng = _rng(seed, 1)
    G = rng.standard_normal((n, 3, 3))
    Qm, Rm = np.linalg.qr(G)
    sgn = np.sign(np.diagonal(Rm, axis1=1, axis2=2))
    sgn[sgn == 0] = 1.0
    Qm = Qm * sgn[:, None, :]
    lam = rng.uniform(0.5, 2.0, size=(n, 3))
    K = np.einsum("nij,nj,nkj->nik", Qm, lam, Qm)
    K = 0.5 * (K + K.transpose(0, 2, 1))
    b = rng.uniform(-1.0, 1.0, size=(n, 3))
    c = rng.uniform(0.0, 1.0, size=n)
    f = rng.uniform(-1.0, 1.0, size=n)
    return dict(K=np.ascontiguousarray(K), b=b, c=c, f=f)


def mixed_degrees(n: int, seed: int, probs=MIXED_PROBS) -> np.ndarray:
    """Degrees p in 1..7 drawn per element with ``probs``, shuffled."""
    rng = _rng(seed, 2)
    counts = rng.multinomial(n, probs)
    deg = np.repeat(np.arange(1, len(probs) + 1, dtype=np.int32), counts)
    rng.shuffle(deg)
    return deg


def sample_points(geom: np.ndarray, degrees) -> np.ndarray:
    """(p+1)^3 sample positions per element (one per quadrature slot): an
    equispaced midpoint lattice of the unit square folded onto the triangle,
    times equispaced heights, placed by vertex interpolation.  These are not
    the quadrature nodes; they only give the per-slot fields a smooth spatial
    structure.  Returns [sum (p_e+1)^3, 3]."""
    geom = np.asarray(geom)
    degs = np.broadcast_to(np.asarray(degrees), (geom.shape[0],))
    out = []
    for p in np.unique(degs):
        idx = np.nonzero(degs == p)[0]
        m = int(p) + 1
        t = (np.arange(m) + 0.5) / m
        zz, bb, aa = np.meshgrid(2 * t - 1, t, t, indexing="ij")
        s2 = bb.reshape(-1)
        s1 = (aa * (1 - bb)).reshape(-1)
        z = zz.reshape(-1)
        lam = np.stack([1 - s1 - s2, s1, s2], axis=1)
        wts = np.concatenate([lam * (0.5 * (1 - z))[:, None], lam * (0.5 * (1 + z))[:, None]], axis=1)
        out.append((idx, np.einsum("qa,nak->nqk", wts, geom[idx])))
    q_counts = (degs.astype(np.int64) + 1) ** 3
    q_off = np.concatenate([[0], np.cumsum(q_counts)])
    res = np.zeros((int(q_off[-1]), 3))
    for idx, pts in out:
        m = pts.shape[1]
        rows = (q_off[idx][:, None] + np.arange(m)[None, :]).reshape(-1)
        res[rows] = pts.reshape(-1, 3)
    return res


def fields_per_point(x: np.ndarray, seed: int) -> dict:
    """Smooth coefficient fields at positions x [m, 3]:
    K(x) = K0 + 0.25 sin(w.x + th) I (K0 SPD, eigenvalues in [0.75, 1.75]),
    b_i(x) = sin(w_i.x + th_i), c(x) = (1 + cos(w_c.x))/2, f(x) = sin(w_f.x),
    frequencies w ~ U[1, 4]^3, phases ~ U[0, 2 pi]."""
    rng = _rng(seed, 3)
    G = rng.standard_normal((3, 3))
    Qm, Rm = np.linalg.qr(G)
    Qm = Qm * np.sign(np.diag(Rm))[None, :]
    K0 = Qm @ np.diag(rng.uniform(0.75, 1.75, size=3)) @ Qm.T
    K0 = 0.5 * (K0 + K0.T)
    wK = rng.uniform(1, 4, size=3)
    thK = rng.uniform(0, 2 * np.pi)
    wb = rng.uniform(1, 4, size=(3, 3))
    thb = rng.uniform(0, 2 * np.pi, size=3)
    wc = rng.uniform(1, 4, size=3)
    wf = rng.uniform(1, 4, size=3)
    m = x.shape[0]
    K = np.broadcast_to(K0, (m, 3, 3)) + (0.25 * np.sin(x @ wK + thK))[:, None, None] * np.eye(3)
    b = np.sin(x @ wb.T + thb[None, :])
    c = 0.5 * (1 + np.cos(x @ wc))
    f = np.sin(x @ wf)
    return dict(K=np.ascontiguousarray(K), b=np.ascontiguousarray(b), c=c, f=f)


def workload(name: str, n_max: int | None = None) -> dict:
    """Build one named workload: dict(geom, degree (int32 [n]) or p, K, b,
    c, f, per_qp).  ``n_max`` truncates to the first n_max elements (same
    seeds, so a truncated workload is a prefix of the full one)."""
    cfg = WORKLOADS[name]
    nx, ny, nz = cfg["grid"]
    geom = prism_mesh(nx, ny, nz, cfg["jitter"], cfg["seed"])
    n = geom.shape[0]
    if cfg["p"] is None:
        degree = mixed_degrees(n, cfg["seed"])
    else:
        degree = np.full(n, cfg["p"], dtype=np.int32)
    coef = None if name == "diff" else coefficients(n, cfg["seed"])
    if coef is not None and cfg.get("symmetric"):
        coef["b"] = np.zeros_like(coef["b"])
    if n_max is not None and n_max < n:
        geom = geom[:n_max]
        degree = degree[:n_max]
        if coef is not None:
            coef = {k: np.ascontiguousarray(v[:n_max]) for k, v in coef.items()}
        n = n_max
    out = dict(geom=np.ascontiguousarray(geom), degree=degree, p=cfg["p"], name=name)
    if name == "diff":
        x = sample_points(geom, degree)
        out.update(fields_per_point(x, cfg["seed"]))
        out["per_qp"] = True
    else:
        out.update(coef)
        out["per_qp"] = False
    return out


def dof_map(w: dict, shared: str = "vertex") -> tuple[np.ndarray, int]:
    """Element-to-global numbering for assembly of workload ``w``: int64
    l2g in the load-vector layout (element e's N_sh(p_e) numbers follow
    those of the elements before it) and the number of global functions.

    ``shared="vertex"``: the first 6 local functions of an element take the
    numbers of its 6 mesh vertices (numbered compactly over the vertices the
    elements use), the others are private, numbered after all vertices in
    element order.  The modal basis has no vertex functions, so this is a
    synthetic sharing pattern; it gives assembly the neighbourhood structure
    of the prism mesh (a vertex is shared by up to 12 prisms).
    ``shared="none"``: every function private (block-diagonal matrix)."""
    cfg = WORKLOADS[w["name"]]
    degree = np.asarray(w["degree"], dtype=np.int64)
    n = len(degree)
    s = (degree + 1) ** 2 * (degree + 2) // 2
    if shared == "none":
        return np.arange(int(s.sum()), dtype=np.int64), int(s.sum())
    if shared != "vertex":
        raise ValueError(shared)
    pv = _prism_vertices(*cfg["grid"])[:n]
    used, vert = np.unique(pv.reshape(-1), return_inverse=True)
    vert = vert.reshape(n, 6)
    n_vert = len(used)
    priv = s - 6
    pstart = n_vert + np.concatenate([[0], np.cumsum(priv)[:-1]])
    l2g = np.empty(int(s.sum()), dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(s)[:-1]])
    for e in range(n):
        o = off[e]
        l2g[o:o + 6] = vert[e]
        l2g[o + 6:o + s[e]] = pstart[e] + np.arange(priv[e])
    return l2g, int(n_vert + priv.sum())


def loss_weights(n_total: int, seed: int) -> np.ndarray:
    """u ~ N(0, 1) FP64 for the loss L = sum_e u_e^T A_e u_e - u_e^T b_e."""
    return _rng(seed, 4).standard_normal(n_total)
