"""Element-by-element and record-by-record comparisons of gradients, and the
selection of the worst-conditioned elements of a mesh (test helpers; no
arithmetic of the method beyond the prism's Jacobian used to rank elements).
"""
from __future__ import annotations

import numpy as np

GRAD_NAMES = ("geom", "K", "b", "c", "f")
GRAD_WIDTHS = (18, 9, 3, 1, 1)


def grad_errors(got, want, n_elem, per_qp, nq_of_elem):
    """Per gradient array: (per-element relative Frobenius errors, per-record
    relative errors).  The per-element errors cover the arrays with a vector
    per element (the 18 vertex coordinates; the records of all points of an
    element for per-point coefficients); for per-element coefficients the
    element's record is checked as a record (an empty element array is
    returned), because one scalar per element (c, f) can cancel to far below
    its neighbours' size.

    got, want: sequences of 5 arrays (g_geom [n,6,3], gK, gb, gc, gf in the
    input layouts).  nq_of_elem: int array [n_elem], records per element for
    per-point coefficients (ignored otherwise).

    A record is one row of a coefficient array (9 values of K, 3 of b, 1 of c,
    1 of f) or one element's 18 vertex coordinates.  Its error is
    ||got_r - want_r|| / max(||want_r||, rms_g), where rms_g is the RMS of
    ||want_r|| over the records of the same element (per-point coefficients)
    or of the whole batch (per-element coefficients, vertex gradients): a
    record that cancels to almost nothing is measured against its
    neighbours' size, not against zero.
    """
    out = {}
    q_off = np.concatenate([[0], np.cumsum(np.asarray(nq_of_elem, dtype=np.int64))]) if per_qp else None
    for name, width, g, w in zip(GRAD_NAMES, GRAD_WIDTHS, got, want):
        g = np.asarray(g, dtype=np.float64).reshape(-1, width)
        w = np.asarray(w, dtype=np.float64).reshape(-1, width)
        assert g.shape == w.shape, (name, g.shape, w.shape)
        err = np.linalg.norm(g - w, axis=1)
        mag = np.linalg.norm(w, axis=1)
        if name != "geom" and per_qp:
            # records of element e: q_off[e] .. q_off[e+1]
            elem_of_rec = np.repeat(np.arange(n_elem), np.diff(q_off))
            ss = np.bincount(elem_of_rec, weights=mag * mag, minlength=n_elem)
            cnt = np.bincount(elem_of_rec, minlength=n_elem)
            rms = np.sqrt(ss / np.maximum(cnt, 1))[elem_of_rec]
            e_num = np.sqrt(np.bincount(elem_of_rec, weights=err * err, minlength=n_elem))
            e_den = np.sqrt(ss)
        else:
            rms = np.full_like(mag, np.sqrt(np.mean(mag * mag)) if len(mag) else 0.0)
            e_num, e_den = (err, mag) if name == "geom" else (np.zeros(0), np.zeros(0))
        rec = err / np.maximum(np.maximum(mag, rms), 1e-300)
        elem = e_num / np.maximum(e_den, 1e-300 + 1e-3 * (np.sqrt(np.mean(e_den * e_den)) if len(e_den) else 0.0))
        out[name] = (elem, rec)
    return out


def assert_grads_close(got, want, n_elem, per_qp, nq_of_elem, tol_elem, tol_rec, where=""):
    """Every element's relative Frobenius error below tol_elem and every
    record's error below tol_rec, for all five gradient arrays."""
    errs = grad_errors(got, want, n_elem, per_qp, nq_of_elem)
    for name, (elem, rec) in errs.items():
        if len(elem):
            ie = int(np.argmax(elem))
            assert elem[ie] < tol_elem, (where, name, "element", ie, float(elem[ie]))
        ir = int(np.argmax(rec))
        assert rec[ir] < tol_rec, (where, name, "record", ir, float(rec[ir]))
    return errs


def prism_jacobian_stats(geom, pts, chunk=2048):
    """For every element of a bilinear-prism batch: the smallest det J over
    the points and the largest ||J||_F ||J^-1||_F over the points.

    geom [n, 6, 3] (bottom 0, 1, 2 at zeta = -1, vertex a+3 above a); pts
    [m, >=3] reference points (xi1, xi2, zeta).  J's columns are the
    derivatives of x = sum_a lambda_a(xi) ((1-zeta)/2 X_a + (1+zeta)/2 X_a+3)
    by xi1, xi2 and zeta."""
    geom = np.asarray(geom, dtype=np.float64)
    xi1, xi2, z = pts[:, 0], pts[:, 1], pts[:, 2]
    lo, hi = (1 - z) / 2, (1 + z) / 2
    n = geom.shape[0]
    min_det = np.empty(n)
    max_cond = np.empty(n)
    for s in range(0, n, chunk):
        X = geom[s:s + chunk]
        P, Q = X[:, :3], X[:, 3:]
        c1 = lo[None, :, None] * (P[:, 1] - P[:, 0])[:, None, :] + hi[None, :, None] * (Q[:, 1] - Q[:, 0])[:, None, :]
        c2 = lo[None, :, None] * (P[:, 2] - P[:, 0])[:, None, :] + hi[None, :, None] * (Q[:, 2] - Q[:, 0])[:, None, :]
        lam = np.stack([1 - xi1 - xi2, xi1, xi2], axis=1)  # [m, 3]
        c3 = 0.5 * np.einsum("ma,nak->nmk", lam, Q - P)
        J = np.stack([c1, c2, c3], axis=-1)  # [n, m, 3 (x), 3 (column)]
        det = np.linalg.det(J)
        inv = np.linalg.inv(J)
        cond = np.linalg.norm(J, axis=(2, 3)) * np.linalg.norm(inv, axis=(2, 3))
        min_det[s:s + chunk] = det.min(axis=1)
        max_cond[s:s + chunk] = cond.max(axis=1)
    return min_det, max_cond


def worst_conditioned(geom, pts, k=64):
    """Indices (sorted, unique) of the k elements with the smallest min det J
    and the k with the largest max ||J|| ||J^-1||."""
    md, mc = prism_jacobian_stats(geom, pts)
    return np.unique(np.concatenate([np.argsort(md)[:k], np.argsort(-mc)[:k]]))
