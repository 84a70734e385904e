"""The FP64 oracle against facts it does not compute itself (CPU only)."""
import json
import os

import numpy as np
import pytest

import oracle
import oracle_pins as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name,fn", P.ALL_PINS, ids=[n for n, _ in P.ALL_PINS])
def test_pin(name, fn):
    fn()


def test_table_sizes_match_paper():
    """Table 1 / Table 2 (shape-function counts and stored sizes per p)."""
    with open(os.path.join(GOLDEN, "table2_sizes.json")) as fh:
        g = json.load(fh)
    for i, p in enumerate(g["p"]):
        s = oracle.nsh(p)
        assert 4 * s == g["phi_and_grad_per_point"][i]
        assert s * s == g["element_matrix"][i]
        pts = oracle.quadrature(p)
        assert pts.shape[0] == (p + 1) ** 3
        phi, dphi = oracle.basis(p, pts[:2, :3])
        assert phi.shape[1] == s and dphi.shape[1:] == (s, 3)


@pytest.mark.parametrize("p", range(1, 8))
def test_orthonormal_all_degrees(p):
    P.pin_orthonormal(p)


@pytest.mark.parametrize("p", [2, 5, 7])
def test_mass_affine_high_p(p):
    P.pin_mass_affine(p)


@pytest.mark.parametrize("p", [4, 7])
def test_volume_high_p(p):
    P.pin_volume(p)


def test_per_point_constant_equals_per_element():
    """Per-point coefficients that are constant reproduce per-element mode."""
    rng = np.random.default_rng(3)
    p, n = 2, 3
    geom = np.stack([P.distorted_prism(rng) for _ in range(n)])
    K = np.stack([P.spd(rng) for _ in range(n)])
    b = rng.uniform(-1, 1, (n, 3))
    c = rng.uniform(0, 1, n)
    f = rng.uniform(-1, 1, n)
    A1, b1, _, _ = oracle.integrate(geom, K, b, c, f, p=p)
    q = oracle.nq(p)
    A2, b2, _, _ = oracle.integrate(geom, np.repeat(K, q, 0), np.repeat(b, q, 0),
                                    np.repeat(c, q), np.repeat(f, q), p=p, per_qp=True)
    assert P.rel(A2, A1) < 1e-14 and P.rel(b2, b1) < 1e-14


def test_mixed_degree_layout_matches_single_degree_calls():
    """A mixed-degree batch equals per-degree batches placed at its offsets."""
    rng = np.random.default_rng(4)
    degs = np.array([1, 3, 2, 1, 3], dtype=np.int32)
    n = len(degs)
    geom = np.stack([P.distorted_prism(rng) for _ in range(n)])
    K = np.stack([P.spd(rng) for _ in range(n)])
    b = rng.uniform(-1, 1, (n, 3))
    c = rng.uniform(0, 1, n)
    f = rng.uniform(-1, 1, n)
    A, bv, st, (Ao, bo, _) = oracle.integrate(geom, K, b, c, f, degree=degs)
    for e in range(n):
        p = int(degs[e])
        s = oracle.nsh(p)
        A1, b1, _, _ = oracle.integrate(geom[e:e + 1], K[e:e + 1], b[e:e + 1], c[e:e + 1], f[e:e + 1], p=p)
        assert np.array_equal(A[Ao[e]:Ao[e] + s * s], A1)
        assert np.array_equal(bv[bo[e]:bo[e] + s], b1)


def test_threads_do_not_change_bits():
    rng = np.random.default_rng(5)
    n = 17
    geom = np.stack([P.distorted_prism(rng) for _ in range(n)])
    K = np.stack([P.spd(rng) for _ in range(n)])
    b = rng.uniform(-1, 1, (n, 3))
    c = rng.uniform(0, 1, n)
    f = rng.uniform(-1, 1, n)
    A1, b1, _, _ = oracle.integrate(geom, K, b, c, f, p=2, nthreads=1)
    A4, b4, _, _ = oracle.integrate(geom, K, b, c, f, p=2, nthreads=4)
    assert np.array_equal(A1, A4) and np.array_equal(b1, b4)


def test_golden_elements_reproduce():
    """Stored oracle values (written by tests/golden/make_golden.py) are
    reproduced to rounding level on this machine."""
    with open(os.path.join(GOLDEN, "oracle_elements.json")) as fh:
        g = json.load(fh)
    geom = np.array(g["geom"])
    for p in (1, 2):
        A, bv, st, _ = oracle.integrate(geom, np.array(g["K"]), np.array(g["b"]),
                                        np.array(g["c"]), np.array(g["f"]), p=p)
        assert P.rel(A, np.array([float(x) for x in g[f"A_p{p}"]])) < 1e-14
        assert P.rel(bv, np.array([float(x) for x in g[f"b_p{p}"]])) < 1e-14
