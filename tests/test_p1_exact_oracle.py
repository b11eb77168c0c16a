"""The order-1 exact-reference-matrix oracle (the paper's P1 precomputation,
Sec. 4.2) pinned to textbook element matrices and to the quadrature oracle."""
import numpy as np
import pytest

import oracle
from paper_2605_14035_gb300.inputs import meshes, quadrature


def _dense(rp, ci, v, n):
    D = np.zeros((n, n))
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = v
    return D


def test_reference_elements():
    # unit right triangle: M = |T|/12 (1 + delta), A the classical 5-point-stencil element
    rp, ci, M, A = oracle.p1_exact(np.array([[0.0, 0], [1, 0], [0, 1]]), np.array([[0, 1, 2]]), 2)
    assert np.allclose(_dense(rp, ci, M, 3) * 24, [[2, 1, 1], [1, 2, 1], [1, 1, 2]], atol=1e-15)
    assert np.allclose(_dense(rp, ci, A, 3), [[1, -0.5, -0.5], [-0.5, 0.5, 0], [-0.5, 0, 0.5]], atol=1e-15)
    # unit tetrahedron: M = |T| (1 + delta) / 20, |T| = 1/6
    rp, ci, M, A = oracle.p1_exact(np.vstack([np.zeros(3), np.eye(3)]), np.array([[0, 1, 2, 3]]), 3)
    assert np.allclose(_dense(rp, ci, M, 4) * 120, 1 + np.eye(4), atol=1e-14)
    Ad = _dense(rp, ci, A, 4)
    assert np.allclose(Ad[1:, 1:], np.eye(3) / 6, atol=1e-15) and np.allclose(Ad[0], [0.5, -1 / 6, -1 / 6, -1 / 6])
    # a segment of length L in R^3: M = L/6 [[2,1],[1,2]], A = [[1,-1],[-1,1]] / L
    x = np.array([[0.3, -1.0, 2.0], [1.5, 0.6, 2.9]])
    L = np.linalg.norm(x[1] - x[0])
    rp, ci, M, A = oracle.p1_exact(x, np.array([[0, 1]]), 1)
    assert np.allclose(_dense(rp, ci, M, 2), L / 6 * np.array([[2, 1], [1, 2]]), atol=1e-15)
    assert np.allclose(_dense(rp, ci, A, 2), np.array([[1, -1], [-1, 1]]) / L, atol=1e-14)


def test_triangle_stiffness_is_scale_and_rotation_invariant():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, 2))
    c, s = np.cos(0.7), np.sin(0.7)
    y = 3.5 * x @ np.array([[c, -s], [s, c]]).T + 1.0
    e = np.array([[0, 1, 2]])
    _, _, M1, A1 = oracle.p1_exact(x, e, 2)
    _, _, M2, A2 = oracle.p1_exact(y, e, 2)
    assert np.allclose(A1, A2, atol=1e-13) and np.allclose(M2, 3.5 ** 2 * M1, rtol=1e-13)


@pytest.mark.parametrize("kind", ["sphere", "disk", "cube", "curve"])
def test_matches_the_quadrature_oracle(kind):
    """The degree-2 rules integrate order-1 M and A exactly on affine elements."""
    if kind == "sphere":
        (x, e), d, r = meshes.icosphere(2, 1), 2, quadrature.tri_3pt_deg2()
    elif kind == "disk":
        (x, e), d, r = meshes.hex_disk(4, 1), 2, quadrature.tri_3pt_deg2()
    elif kind == "cube":
        (x, e), d, r = meshes.kuhn_cube_p2(3, order=1), 3, quadrature.tet_4pt_deg2()
    else:
        t = np.linspace(0, 2 * np.pi, 41)[:-1]
        x = np.stack([np.cos(t), np.sin(t), 0.3 * np.sin(3 * t)], axis=1)
        e = np.stack([np.arange(40), (np.arange(40) + 1) % 40], axis=1)
        d, r = 1, quadrature.gauss_interval(2)
    rp, ci, M, A = oracle.p1_exact(x, e, d)
    rp2, ci2, M2, A2, _ = oracle.assemble(x, e, d, 1, r.xi, r.w)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    assert np.abs(M - M2).max() <= 1e-14 * np.abs(M).max()
    assert np.abs(A - A2).max() <= 1e-13 * np.abs(A).max()
