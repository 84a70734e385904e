"""Pins of the FP64 oracle against facts that do not come from the oracle.

Every check here compares the oracle with something it does not compute
itself: a library routine (numpy's Gauss-Legendre, scipy's Gauss-Jacobi), a
closed form (monomial integrals on the triangle, the element volume by the
divergence theorem), an invariant (rigid motions, scaling laws, symmetry,
the constant function's null space), an identity with a closed-form answer
(linear functions against the convection and diffusion terms), central finite
differences, or a brute-force high-order rule with a Jacobian computed here.

Each ``pin_*`` function raises AssertionError on a mismatch.  The same
functions run against deliberately broken builds of the oracle in
``test_oracle_mutations.py`` to show that a plausible mistake anywhere in
the oracle fails at least one pin.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import roots_jacobi

import oracle

# reference prism vertices in (xi1, xi2, zeta): bottom 0,1,2 then top 3,4,5
REF_VERTS = np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1],
                      [0, 0, 1], [1, 0, 1], [0, 1, 1]], dtype=np.float64)


# ---------------------------------------------------------------------------
# independent rules and geometry written here (not the oracle's)
# ---------------------------------------------------------------------------

def prism_rule(n: int):
    """Gauss-Legendre in u and zeta, Gauss-Jacobi(1, 0) in v (the (1-v)
    collapse factor is the Jacobi weight), folded onto the triangle:
    a different rule from the oracle's.  Returns points [m,3], weights [m]."""
    u, wu = leggauss(n)
    v, wv = roots_jacobi(n, 1.0, 0.0)
    z, wz = leggauss(n)
    U, V, Z = np.meshgrid(u, v, z, indexing="ij")
    W = wu[:, None, None] * wv[None, :, None] * wz[None, None, :] / 8.0
    xi1 = (1 + U) * (1 - V) / 4
    xi2 = (1 + V) / 2
    return np.stack([xi1.ravel(), xi2.ravel(), Z.ravel()], 1), W.ravel()


def affine_prism(rng, x0=None, M=None):
    """Vertices X_a = x0 + M r_a of an affine prism (det M > 0)."""
    if M is None:
        M = np.eye(3) * 0.3 + 0.08 * rng.standard_normal((3, 3))
        if np.linalg.det(M) < 0:
            M[:, 0] *= -1
    if x0 is None:
        x0 = rng.uniform(-1, 1, 3)
    return x0[None, :] + REF_VERTS @ M.T, M, x0


def distorted_prism(rng, amount=0.25):
    """A bilinear prism: reference prism scaled, vertices moved independently."""
    base = REF_VERTS * np.array([0.5, 0.5, 0.25])
    X = base + amount * 0.25 * rng.uniform(-1, 1, (6, 3))
    return X


def spd(rng):
    G = rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(G)
    return Q @ np.diag(rng.uniform(0.5, 2.0, 3)) @ Q.T


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def single(X, K, bb, c, f, p):
    """Oracle on one element with per-element coefficients: (A [nsh,nsh], b)."""
    s = oracle.nsh(p)
    A, bv, st, _ = oracle.integrate(np.asarray(X)[None], np.asarray(K, float)[None],
                                    np.asarray(bb, float)[None], np.array([c], float),
                                    np.array([f], float), p=p)
    assert st[0] == 0, f"status {st[0]}"
    return A.reshape(s, s), bv


def volume_divergence(X):
    """Volume of a bilinear prism by the divergence theorem, V = 1/3 int x.n,
    with the planar caps in closed form and each bilinear side patch
    integrated by a 2x2 Gauss rule (exact for its bilinear integrand)."""
    P, Q = X[:3], X[3:]
    vol = 0.0
    vol += np.dot(P.mean(0), -0.5 * np.cross(P[1] - P[0], P[2] - P[0]))
    vol += np.dot(Q.mean(0), 0.5 * np.cross(Q[1] - Q[0], Q[2] - Q[0]))
    g, gw = leggauss(2)
    s_pts, s_w = (g + 1) / 2, gw / 2
    for a, b in ((0, 1), (1, 2), (2, 0)):
        for s, ws in zip(s_pts, s_w):
            for t, wt in zip(s_pts, s_w):
                x = (1 - s) * (1 - t) * P[a] + s * (1 - t) * P[b] + s * t * Q[b] + (1 - s) * t * Q[a]
                xs = (1 - t) * (P[b] - P[a]) + t * (Q[b] - Q[a])
                xt = (1 - s) * (Q[a] - P[a]) + s * (Q[b] - P[b])
                vol += ws * wt * np.dot(x, np.cross(xs, xt))
    return vol / 3.0


# ---------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------

def pin_gauss():
    """Gauss-Legendre nodes/weights equal numpy's leggauss; sum w = 2."""
    for n in range(1, 9):
        x, w = oracle.gauss_legendre(n)
        xr, wr = leggauss(n)
        assert np.max(np.abs(x - xr)) < 1e-14, (n, x, xr)
        assert np.max(np.abs(w - wr)) < 1e-14, (n, w, wr)
        assert abs(w.sum() - 2.0) < 1e-14


def pin_duffy_monomials(p):
    """sum_q w xi1^a xi2^b zeta^k = a! b!/(a+b+2)! * int zeta^k for a+b <= 2p,
    k <= 2p+1 (exactness of the collapsed rule, closed form)."""
    pts = oracle.quadrature(p)
    x1, x2, z, w = pts.T
    assert pts.shape[0] == (p + 1) ** 3
    for a in range(2 * p + 1):
        for b in range(2 * p + 1 - a):
            for k in (0, 1, 2 * p, 2 * p + 1):
                exact_t = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                exact_z = (1 - (-1) ** (k + 1)) / (k + 1)
                got = np.sum(w * x1 ** a * x2 ** b * z ** k)
                assert abs(got - exact_t * exact_z) < 1e-14, (p, a, b, k, got, exact_t * exact_z)


def pin_orthonormal(p):
    """Gram matrix of the basis under an independent rule is the identity."""
    pts, w = prism_rule(p + 3)
    phi, _ = oracle.basis(p, pts)
    G = (phi * w[:, None]).T @ phi
    err = np.max(np.abs(G - np.eye(G.shape[0])))
    assert err < 1e-11, (p, err)


def pin_gradient_fd(p, seed=11):
    """Reference gradients equal central finite differences of the values."""
    rng = np.random.default_rng(seed)
    for _ in range(4):
        s2 = rng.uniform(0.05, 0.8)
        s1 = rng.uniform(0.05, 0.9) * (1 - s2)
        z = rng.uniform(-0.9, 0.9)
        x = np.array([s1, s2, z])
        _, d = oracle.basis(p, x)
        h = 1e-6
        for l in range(3):
            e = np.zeros(3)
            e[l] = h
            fp, _ = oracle.basis(p, x + e)
            fm, _ = oracle.basis(p, x - e)
            fd = (fp[0] - fm[0]) / (2 * h)
            scale = max(1.0, np.max(np.abs(d[0, :, l])))
            assert np.max(np.abs(fd - d[0, :, l])) < 1e-6 * scale, (p, l)


def _monomial_matrix(pts, p, tri_deg, z_deg):
    cols = []
    for k in range(z_deg + 1):
        for d in range(tri_deg + 1):
            for a in range(d + 1):
                cols.append(pts[:, 0] ** a * pts[:, 1] ** (d - a) * pts[:, 2] ** k)
    return np.stack(cols, 1)


def pin_span_and_order(p, seed=12):
    """Each phi_i lies in P_d(triangle) x P_k(zeta) with (d, k) given by the
    basis order index = k*T_p + t, t over total degree d ascending (and not
    in the smaller spaces); phi_0 = 1; the m-index of psi_{m,n} is its degree
    in xi1 along lines of constant xi2; a fixed sign convention holds."""
    rng = np.random.default_rng(seed)
    m_pts = 400
    s2 = rng.uniform(0.0, 0.9, m_pts)
    s1 = rng.uniform(0, 1, m_pts) * (1 - s2)
    z = rng.uniform(-1, 1, m_pts)
    pts = np.stack([s1, s2, z], 1)
    phi, _ = oracle.basis(p, pts)
    assert np.max(np.abs(phi[:, 0] - 1.0)) < 1e-13
    T = (p + 1) * (p + 2) // 2
    tri = [(d - n, n) for d in range(p + 1) for n in range(d + 1)]
    for i in range(phi.shape[1]):
        k, t = divmod(i, T)
        m, n = tri[t]
        d = m + n
        V = _monomial_matrix(pts, p, d, k)
        coef, *_ = np.linalg.lstsq(V, phi[:, i], rcond=None)
        res = np.linalg.norm(V @ coef - phi[:, i]) / np.linalg.norm(phi[:, i])
        assert res < 1e-9, (p, i, "not in P_d x P_k", res)
        # strictly of degree (d, k): fails in the smaller spaces
        for (dd, kk) in ((d - 1, k), (d, k - 1)):
            if dd < 0 or kk < 0:
                continue
            V2 = _monomial_matrix(pts, p, dd, kk)
            c2, *_ = np.linalg.lstsq(V2, phi[:, i], rcond=None)
            r2 = np.linalg.norm(V2 @ c2 - phi[:, i]) / np.linalg.norm(phi[:, i])
            assert r2 > 1e-3, (p, i, "degree too low", dd, kk)
    # degree m in xi1 along a horizontal line
    for t, (m, n) in enumerate(tri):
        xs2 = 0.3
        xs1 = np.linspace(0.01, 0.69, 2 * p + 3)
        pl = np.stack([xs1, np.full_like(xs1, xs2), np.full_like(xs1, 0.2)], 1)
        ph, _ = oracle.basis(p, pl)
        y = ph[:, t]
        cm = np.polyfit(xs1, y, m)
        assert np.max(np.abs(np.polyval(cm, xs1) - y)) < 1e-8 * max(1, np.max(np.abs(y))), (p, m, n)
        if m >= 1:
            cm1 = np.polyfit(xs1, y, m - 1)
            assert np.max(np.abs(np.polyval(cm1, xs1) - y)) > 1e-6, (p, m, n)
    # sign convention: positive near the collapsed vertex along the hypotenuse, at zeta = 1
    s = 0.999
    ph, _ = oracle.basis(p, np.array([[1 - s, s, 1.0]]))
    assert np.all(ph[0] > 0), (p, ph[0])


def pin_mass_affine(p, seed=13):
    """Affine prism, K = 0, b = 0, c = 1: A = det(M) I (orthonormal basis,
    reference volume 1)."""
    rng = np.random.default_rng(seed)
    X, M, _ = affine_prism(rng)
    A, _ = single(X, np.zeros((3, 3)), np.zeros(3), 1.0, 0.0, p)
    err = np.max(np.abs(A - np.linalg.det(M) * np.eye(A.shape[0])))
    assert err < 1e-14 * max(1.0, np.linalg.det(M)) * 10, (p, err)


def pin_volume(p, seed=14):
    """Distorted prism: A_00 with c = 1 and b_0 with f = 1 both equal the
    volume from the divergence theorem."""
    rng = np.random.default_rng(seed)
    for _ in range(3):
        X = distorted_prism(rng)
        vol = volume_divergence(X)
        A, bv = single(X, np.zeros((3, 3)), np.zeros(3), 1.0, 1.0, p)
        assert abs(A[0, 0] - vol) < 1e-13 * abs(vol) * 10, (p, A[0, 0], vol)
        assert abs(bv[0] - vol) < 1e-13 * abs(vol) * 10, (p, bv[0], vol)


def pin_constant_null(p, seed=15):
    """Diffusion only: the constant function phi_0 is in the null space from
    both sides (A e0 = 0, e0^T A = 0); with convection only, A e0 = 0."""
    rng = np.random.default_rng(seed)
    X = distorted_prism(rng)
    A, _ = single(X, spd(rng), np.zeros(3), 0.0, 0.0, p)
    sc = np.max(np.abs(A))
    assert np.max(np.abs(A[:, 0])) < 1e-13 * sc and np.max(np.abs(A[0, :])) < 1e-13 * sc
    A, _ = single(X, np.zeros((3, 3)), rng.uniform(-1, 1, 3), 0.0, 0.0, p)
    assert np.max(np.abs(A[:, 0])) < 1e-13 * np.max(np.abs(A))


def pin_symmetry(p, seed=16):
    """Symmetric K, b = 0: A = A^T; with b != 0 it is not."""
    rng = np.random.default_rng(seed)
    X = distorted_prism(rng)
    K = spd(rng)
    A, _ = single(X, K, np.zeros(3), 0.7, 0.0, p)
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))
    A, _ = single(X, K, np.array([0.5, -0.3, 0.8]), 0.7, 0.0, p)
    assert np.max(np.abs(A - A.T)) > 1e-6 * np.max(np.abs(A))


def pin_rigid_motion(p, seed=17):
    """Rotating and translating the element with K -> R K R^T, b -> R b
    leaves A and b_e unchanged."""
    rng = np.random.default_rng(seed)
    X = distorted_prism(rng)
    K = spd(rng)
    bb = rng.uniform(-1, 1, 3)
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    t = rng.uniform(-2, 2, 3)
    A1, b1 = single(X, K, bb, 0.4, 0.6, p)
    A2, b2 = single(X @ R.T + t, R @ K @ R.T, R @ bb, 0.4, 0.6, p)
    assert rel(A2, A1) < 1e-12 and rel(b2, b1) < 1e-12, (p, rel(A2, A1))


def pin_scaling(p, seed=18):
    """Scaling the element by s scales diffusion by s, convection by s^2,
    reaction and load by s^3."""
    rng = np.random.default_rng(seed)
    X = distorted_prism(rng)
    s = 1.7
    K = spd(rng)
    bb = rng.uniform(-1, 1, 3)
    Ad, _ = single(X, K, np.zeros(3), 0.0, 0.0, p)
    Ad2, _ = single(s * X, K, np.zeros(3), 0.0, 0.0, p)
    Ac, _ = single(X, np.zeros((3, 3)), bb, 0.0, 0.0, p)
    Ac2, _ = single(s * X, np.zeros((3, 3)), bb, 0.0, 0.0, p)
    Ar, br = single(X, np.zeros((3, 3)), np.zeros(3), 0.8, 0.6, p)
    Ar2, br2 = single(s * X, np.zeros((3, 3)), np.zeros(3), 0.8, 0.6, p)
    assert rel(Ad2, s * Ad) < 1e-12
    assert rel(Ac2, s ** 2 * Ac) < 1e-12
    assert rel(Ar2, s ** 3 * Ar) < 1e-12 and rel(br2, s ** 3 * br) < 1e-12


def _coef_of_linear(p, k, M, x0):
    """Coefficients of x_k = x0_k + (M xi)_k in the basis, by L2 projection
    on the reference prism with an independent rule (exact: x_k is in the
    span and the basis is orthonormal there)."""
    pts, w = prism_rule(p + 2)
    phi, _ = oracle.basis(p, pts)
    xk = x0[k] + pts @ M[k]
    return (phi * (w * xk)[:, None]).sum(0)


def pin_convection_identity(p, seed=19):
    """Affine element, convection only: A u = b_k det(M) e_0 where u are the
    coefficients of x_k (int phi_i b.grad x_k = b_k vol delta_i0).  Pins the
    orientation (test i, trial j) and the J^{-T} of the convection term."""
    rng = np.random.default_rng(seed)
    X, M, x0 = affine_prism(rng)
    bb = np.array([0.7, -0.4, 0.9])
    A, _ = single(X, np.zeros((3, 3)), bb, 0.0, 0.0, p)
    for k in range(3):
        u = _coef_of_linear(p, k, M, x0)
        want = np.zeros(A.shape[0])
        want[0] = bb[k] * np.linalg.det(M)
        got = A @ u
        assert np.max(np.abs(got - want)) < 1e-12 * max(1, np.max(np.abs(A)) * np.max(np.abs(u))), (p, k)


def pin_diffusion_identity(p, seed=20):
    """Affine element, non-symmetric K: (A u)_i = det(M) (M^{-1} K e_k) .
    int grad_ref phi_i, u the coefficients of x_k; the reference integral of
    the gradients uses an independent rule."""
    rng = np.random.default_rng(seed)
    X, M, x0 = affine_prism(rng)
    K = spd(rng) + 0.3 * np.array([[0, 1, 0], [-1, 0, 0.5], [0, -0.5, 0]])
    A, _ = single(X, K, np.zeros(3), 0.0, 0.0, p)
    pts, w = prism_rule(p + 2)
    _, dphi = oracle.basis(p, pts)
    gint = np.einsum("q,qil->il", w, dphi)
    Minv = np.linalg.inv(M)
    for k in range(3):
        u = _coef_of_linear(p, k, M, x0)
        want = np.linalg.det(M) * gint @ (Minv @ K[:, k])
        got = A @ u
        assert np.max(np.abs(got - want)) < 1e-11 * max(1, np.max(np.abs(want))), (p, k, np.max(np.abs(got - want)))


def pin_brute_force_affine(p, seed=21):
    """Affine element, constant coefficients: A equals the same weak form
    integrated with an independent high-order rule and a Jacobian computed
    here (the integrand is polynomial there, so both rules are exact)."""
    rng = np.random.default_rng(seed)
    X, M, _ = affine_prism(rng)
    K = spd(rng)
    bb = rng.uniform(-1, 1, 3)
    c, f = 0.6, -0.3
    A, bv = single(X, K, bb, c, f, p)
    pts, w = prism_rule(p + 3)
    phi, dphi = oracle.basis(p, pts)
    det = np.linalg.det(M)
    G = dphi @ np.linalg.inv(M)  # physical gradients: J^{-T} g = (g^T J^{-1})^T
    Aw = (np.einsum("q,qik,kl,qjl->ij", w * det, G, K, G)
          + np.einsum("q,qi,k,qjk->ij", w * det, phi, bb, G)
          + c * np.einsum("q,qi,qj->ij", w * det, phi, phi))
    bw = f * np.einsum("q,qi->i", w * det, phi)
    assert rel(A, Aw) < 1e-12, (p, rel(A, Aw))
    assert rel(bv, bw) < 1e-12


def pin_linearity(p, seed=22):
    """A is linear in (K, b, c) and b_e in f."""
    rng = np.random.default_rng(seed)
    X = distorted_prism(rng)
    K1, K2 = spd(rng), spd(rng)
    b1, b2 = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    A1, v1 = single(X, K1, b1, 0.3, 0.2, p)
    A2, v2 = single(X, K2, b2, 0.5, -0.7, p)
    A3, v3 = single(X, K1 + 2 * K2, b1 + 2 * b2, 1.3, -1.2, p)
    assert rel(A3, A1 + 2 * A2) < 1e-13 and rel(v3, v1 + 2 * v2) < 1e-13


def pin_status(p):
    """An inverted element flags 3 with zero outputs; a NaN input flags 4."""
    rng = np.random.default_rng(23)
    X = distorted_prism(rng)
    Xi = X[[0, 2, 1, 3, 5, 4]]  # mirrored orientation: det J < 0
    geom = np.stack([X, Xi, X])
    K = np.stack([spd(rng)] * 3)
    bb = np.zeros((3, 3))
    c = np.ones(3)
    f = np.ones(3)
    c[2] = np.nan
    A, bv, st, _ = oracle.integrate(geom, K, bb, c, f, p=p)
    s = oracle.nsh(p)
    assert list(st) == [0, oracle.ERR_NEGATIVE_JACOBIAN, oracle.ERR_NONFINITE], st
    assert np.all(A[s * s:] == 0) and np.all(bv[s:] == 0)
    assert np.any(A[:s * s] != 0)


def pin_backward_fd(p, seed=24, per_qp=False):
    """Vertex-coordinate gradient of L = <gA, A> + <gb, b> equals central
    finite differences (step 1e-6) of the forward."""
    rng = np.random.default_rng(seed)
    n = 2
    geom = np.stack([distorted_prism(rng) for _ in range(n)])
    s, q = oracle.nsh(p), oracle.nq(p)
    m = n * q if per_qp else n
    K = np.stack([spd(rng) for _ in range(m)])
    bb = rng.uniform(-1, 1, (m, 3))
    c = rng.uniform(0, 1, m)
    f = rng.uniform(-1, 1, m)
    gA = rng.standard_normal(n * s * s)
    gb = rng.standard_normal(n * s)

    def L(g):
        A, bv, st, _ = oracle.integrate(g, K, bb, c, f, p=p, per_qp=per_qp)
        return float(gA @ A + gb @ bv)

    gX, gK, gbc, gc, gf = oracle.integrate_backward(geom, K, bb, c, f, gA, gb, p=p, per_qp=per_qp)
    h = 1e-6
    fd = np.zeros_like(geom)
    for e in range(n):
        for a in range(6):
            for k in range(3):
                gp = geom.copy()
                gm = geom.copy()
                gp[e, a, k] += h
                gm[e, a, k] -= h
                fd[e, a, k] = (L(gp) - L(gm)) / (2 * h)
    assert rel(gX, fd) < 1e-6, (p, rel(gX, fd))
    # coefficients: L is linear in them, so a finite step is exact
    dK = rng.standard_normal(K.shape)
    db = rng.standard_normal(bb.shape)
    dc = rng.standard_normal(c.shape)
    df = rng.standard_normal(f.shape)
    L0 = L(geom)
    A1, v1, _, _ = oracle.integrate(geom, K + dK, bb + db, c + dc, f + df, p=p, per_qp=per_qp)
    dL = float(gA @ A1 + gb @ v1) - L0
    pred = float(np.sum(gK * dK) + np.sum(gbc * db) + np.sum(gc * dc) + np.sum(gf * df))
    assert abs(dL - pred) < 1e-10 * max(1.0, abs(dL)), (p, dL, pred)


ALL_PINS = [
    ("gauss", lambda: pin_gauss()),
    ("duffy", lambda: [pin_duffy_monomials(p) for p in (1, 3, 7)]),
    ("orthonormal", lambda: [pin_orthonormal(p) for p in (1, 2, 4)]),
    ("gradient_fd", lambda: [pin_gradient_fd(p) for p in (2, 5)]),
    ("span_order", lambda: [pin_span_and_order(p) for p in (1, 3)]),
    ("mass_affine", lambda: [pin_mass_affine(p) for p in (1, 3)]),
    ("volume", lambda: [pin_volume(p) for p in (1, 2)]),
    ("constant_null", lambda: [pin_constant_null(p) for p in (1, 3)]),
    ("symmetry", lambda: [pin_symmetry(p) for p in (2,)]),
    ("rigid_motion", lambda: [pin_rigid_motion(p) for p in (2,)]),
    ("scaling", lambda: [pin_scaling(p) for p in (2,)]),
    ("convection_identity", lambda: [pin_convection_identity(p) for p in (1, 3)]),
    ("diffusion_identity", lambda: [pin_diffusion_identity(p) for p in (1, 3)]),
    ("brute_force_affine", lambda: [pin_brute_force_affine(p) for p in (1, 3)]),
    ("linearity", lambda: [pin_linearity(p) for p in (2,)]),
    ("status", lambda: [pin_status(p) for p in (1,)]),
    ("backward_fd", lambda: [pin_backward_fd(p) for p in (1, 2)]),
    ("backward_fd_per_qp", lambda: [pin_backward_fd(p, per_qp=True) for p in (2,)]),
]
