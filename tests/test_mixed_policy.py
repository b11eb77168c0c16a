"""The conditioning test of the mixed path: a metric quality q = det G / (tr G / d)^d
at or above 4k/(1+k)^2 bounds cond(G) by k (d = 2 exactly, d = 3 as an upper
envelope), so the quality threshold derived from kappa_max never keeps in FP32
an element whose metric is worse conditioned than kappa_max."""
import numpy as np


def _quality(G):
    d = G.shape[-1]
    return np.linalg.det(G) / (np.trace(G, axis1=-2, axis2=-1) / d) ** d


def _q_of_kappa(k):
    return 4 * k / (1 + k) ** 2


def _spd(rng, n, d):
    J = rng.standard_normal((n, d, d)) * np.exp(rng.uniform(-1.5, 1.5, (n, 1, d)))
    return np.einsum("nki,nkj->nij", J, J)


def test_two_dimensional_metric_quality_is_a_function_of_the_condition_number():
    rng = np.random.default_rng(11)
    G = _spd(rng, 2000, 2)
    lam = np.linalg.eigvalsh(G)
    kappa = lam[:, 1] / lam[:, 0]
    np.testing.assert_allclose(_quality(G), _q_of_kappa(kappa), rtol=1e-7)


def test_three_dimensional_quality_bounds_the_condition_number():
    rng = np.random.default_rng(12)
    G = _spd(rng, 5000, 3)
    lam = np.linalg.eigvalsh(G)
    kappa = lam[:, 2] / lam[:, 0]
    q = _quality(G)
    assert np.all(q <= _q_of_kappa(kappa) * (1 + 1e-9))
    # the envelope is reached when the middle eigenvalue is the mean of the outer two
    l1, l3 = rng.uniform(0.1, 1, 100), rng.uniform(1, 50, 100)
    G_env = np.zeros((100, 3, 3))
    G_env[:, 0, 0], G_env[:, 1, 1], G_env[:, 2, 2] = l1, (l1 + l3) / 2, l3
    np.testing.assert_allclose(_quality(G_env), _q_of_kappa(l3 / l1), rtol=1e-12)


def test_threshold_is_monotone_in_kappa():
    k = np.array([1.0, 2.0, 7 + 4 * np.sqrt(3), 64.0, 1e3, 1e6])
    q = _q_of_kappa(k)
    assert q[0] == 1.0 and abs(q[2] - 0.25) < 1e-15 and abs(q[3] - 256 / 4225) < 1e-15
    assert np.all(np.diff(q) < 0)
