"""The seeded input generator: sizes, determinism, prefix property, validity."""
import numpy as np

from paper_1310_1194_gb300 import inputs
import oracle_pins as P


def test_counts_and_determinism():
    w1 = inputs.workload("pr1")
    w2 = inputs.workload("pr1")
    assert w1["geom"].shape == (4096, 6, 3)
    assert np.array_equal(w1["geom"], w2["geom"]) and np.array_equal(w1["K"], w2["K"])
    assert np.all(w1["degree"] == 1)


def test_prefix_property():
    full = inputs.workload("pr1")
    part = inputs.workload("pr1", n_max=100)
    for k in ("geom", "K", "b", "c", "f", "degree"):
        assert np.array_equal(part[k], full[k][:100]), k


def test_spd_and_ranges():
    w = inputs.workload("pr1")
    ev = np.linalg.eigvalsh(w["K"])
    assert ev.min() >= 0.5 - 1e-12 and ev.max() <= 2.0 + 1e-12
    assert np.all(np.abs(w["b"]) <= 1) and np.all((w["c"] >= 0) & (w["c"] <= 1))
    assert np.all(np.abs(w["f"]) <= 1)


def test_mixed_degree_distribution():
    d = inputs.mixed_degrees(200_000, 3)
    frac = np.bincount(d, minlength=8)[1:] / d.size
    assert np.allclose(frac, inputs.MIXED_PROBS, atol=0.005)


def test_strong_jitter_mesh_valid_everywhere():
    """+-25% jitter mesh: the certificate holds, and the volumes computed by
    the divergence theorem sum to the unit cube."""
    geom = inputs.prism_mesh(8, 8, 4, 0.25, seed=5)
    assert inputs._element_valid(geom).all()
    vols = np.array([P.volume_divergence(X) for X in geom])
    assert vols.min() > 0
    # boundary vertices are jittered too, so the union is a perturbed cube
    assert abs(vols.sum() - 1.0) < 0.1


def test_certificate_rejects_inverted():
    X = P.distorted_prism(np.random.default_rng(0))
    assert inputs._element_valid(X[None]).all()
    assert not inputs._element_valid(X[[0, 2, 1, 3, 5, 4]][None]).any()


def test_per_point_fields_shape():
    w = inputs.workload("diff", n_max=10)
    assert w["per_qp"] and w["K"].shape == (10 * 216, 3, 3)
    ev = np.linalg.eigvalsh(w["K"])
    assert ev.min() > 0.4 and ev.max() < 2.1
