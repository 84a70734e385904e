"""The comparison helpers the GPU parity tests use, checked on the CPU: a
planted wrong record or element is caught, identical arrays pass, and the
Jacobian statistics of the reference prism and of a scaled copy are the
known values."""
import numpy as np
import pytest

from parity_util import assert_grads_close, grad_errors, prism_jacobian_stats, worst_conditioned

REF_PRISM = np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], dtype=np.float64)


def _grads(n, q, per_qp, seed):
    rng = np.random.default_rng(seed)
    m = n * q if per_qp else n
    return [rng.standard_normal((n, 6, 3)), rng.standard_normal((m, 3, 3)), rng.standard_normal((m, 3)),
            rng.standard_normal(m), rng.standard_normal(m)]


@pytest.mark.parametrize("per_qp", [False, True])
def test_identical_gradients_pass(per_qp):
    g = _grads(4, 27, per_qp, 1)
    errs = assert_grads_close(g, g, 4, per_qp, np.full(4, 27), 1e-14, 1e-14)
    assert all((len(v[0]) == 0 or v[0].max() == 0) and v[1].max() == 0 for v in errs.values())


@pytest.mark.parametrize("name_idx", range(5))
def test_one_wrong_record_is_caught(name_idx):
    """One record among 4 x 216 off by 1e-4 of the element's size: hidden
    under a batch-wide norm at 1e-6 of 5 elements' worth of records, caught
    record by record."""
    n, q = 5, 216
    want = _grads(n, q, True, 2)
    got = [x.copy() for x in want]
    flat = got[name_idx].reshape(-1)
    flat[7] += 1e-4 * np.sqrt(np.mean(want[name_idx] ** 2))
    errs = grad_errors(got, want, n, True, np.full(n, q))
    elem, rec = errs[("geom", "K", "b", "c", "f")[name_idx]]
    assert rec.max() > 1e-5
    with pytest.raises(AssertionError):
        assert_grads_close(got, want, n, True, np.full(n, q), 1e-3, 1e-5)


def test_record_that_cancels_is_measured_against_its_neighbours():
    n, q = 2, 8
    want = _grads(n, q, True, 3)
    want[3][5] = 1e-12  # a c-record that is almost zero
    got = [x.copy() for x in want]
    got[3][5] += 1e-9  # tiny absolute error on it
    elem, rec = grad_errors(got, want, n, True, np.full(n, q))["c"]
    assert rec.max() < 1e-8


def test_reference_prism_jacobian_is_identity():
    pts = np.array([[0.2, 0.3, -0.5], [0.1, 0.1, 0.9], [0.6, 0.2, 0.0]])
    md, mc = prism_jacobian_stats(REF_PRISM[None], pts)
    assert abs(md[0] - 1.0) < 1e-15
    assert abs(mc[0] - 3.0) < 1e-14  # ||I||_F ||I||_F


def test_scaled_and_sheared_prisms_rank_as_expected():
    pts = np.array([[1 / 3, 1 / 3, 0.0], [0.1, 0.8, -0.9]])
    small = REF_PRISM * 0.5  # det J = 1/8 everywhere
    shear = REF_PRISM.copy()
    shear[3:, 0] += 3.0  # top face shifted: J's third column tilted, det unchanged
    geom = np.stack([REF_PRISM, small, shear])
    md, mc = prism_jacobian_stats(geom, pts)
    assert np.allclose(md, [1.0, 0.125, 1.0])
    assert mc[2] > mc[0] and abs(mc[1] - 3.0) < 1e-13
    assert list(worst_conditioned(geom, pts, k=1)) == [1, 2]
