"""Orders 3 and 4 on tetrahedra: the oracle's assembly pinned to exact
integrals over the unit cube, and the order-p node generation of the input
module pinned to the documented node order.

* affine (jittered Kuhn) meshes: for a polynomial u of degree p the nodal
  interpolant is u itself, so u^T M u and u^T A u are the exact integrals of
  u^2 and |grad u|^2 over the cube (tensor Gauss-Legendre, exact here);
* curved meshes (interior nodes moved, boundary faces left flat, so the
  elements still tile the cube): the space holds x, y, z exactly, so with a
  rule exact for det J (degree 3(p-1)) sum M = 1, X^T A X = I, A 1 = 0, and
  with a rule exact for x det J (degree 4p-3), x^T M 1 = 1/2.
"""
import numpy as np
import pytest

import oracle
from paper_2605_14035_gb300.inputs import meshes, quadrature

from test_high_order_oracle import node_alphas


def _cube(p, n=2, jitter=0.1):
    x1, t1 = meshes.kuhn_cube_p2(n, jitter=jitter, order=1)
    return meshes.to_order(x1, t1, p)


def _cube_integral(f, n=12):
    """Tensor Gauss-Legendre over [0, 1]^3 (exact for degree <= 2n - 1 per axis)."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = (g + 1) / 2, w / 2
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return float((f(X, Y, Z) * W).sum())


def _dense(rp, ci, vals, N):
    D = np.zeros((N, N))
    rows = np.repeat(np.arange(N), np.diff(rp))
    np.add.at(D, (rows, ci), vals)
    return D


POLY = {
    3: (lambda x, y, z: x * x * y - 0.5 * z ** 3 + x * y * z + 0.3 * y,
        lambda x, y, z: (2 * x * y + y * z, x * x + x * z + 0.3, -1.5 * z * z + x * y)),
    4: (lambda x, y, z: x * x * y * y - z ** 4 + 0.7 * x * y * z * z + x ** 3 - 0.2 * z,
        lambda x, y, z: (2 * x * y * y + 0.7 * y * z * z + 3 * x * x, 2 * x * x * y + 0.7 * x * z * z,
                         -4 * z ** 3 + 1.4 * x * y * z - 0.2)),
}


@pytest.mark.parametrize("p", [3, 4])
def test_affine_tets_integrate_degree_p_polynomials_exactly(p):
    x, e = _cube(p)
    N = x.shape[0]
    rule = quadrature.collapsed_gauss(3, p + 1)   # degree 2p + 1 >= 2p
    rp, ci, M, A, _ = oracle.assemble(x, e, 3, p, rule.xi, rule.w)
    u_f, g_f = POLY[p]
    u = u_f(x[:, 0], x[:, 1], x[:, 2])
    Md, Ad = _dense(rp, ci, M, N), _dense(rp, ci, A, N)
    mass = _cube_integral(lambda X, Y, Z: u_f(X, Y, Z) ** 2)
    stiff = _cube_integral(lambda X, Y, Z: sum(c ** 2 for c in g_f(X, Y, Z)))
    assert abs(u @ Md @ u - mass) < 1e-12 * mass
    assert abs(u @ Ad @ u - stiff) < 1e-11 * stiff
    assert abs(Md.sum() - 1.0) < 1e-13


def _curved_cube(p, amp=0.005, seed=11):
    x, e = _cube(p)
    on_bnd = np.any((x < 1e-12) | (x > 1 - 1e-12), axis=1)
    rng = np.random.default_rng(meshes.BASE_SEED + seed)
    d = rng.uniform(-amp, amp, x.shape)
    # move only generated (non-vertex) interior nodes, so corners stay affine
    # while edges, faces and cells bend
    move = ~on_bnd & (np.arange(x.shape[0]) >= int(e[:, :4].max()) + 1)
    return x + np.where(move[:, None], d, 0.0), e, move


@pytest.mark.parametrize("p", [3, 4])
def test_curved_tets_tile_the_cube(p):
    x, e, move = _curved_cube(p)
    assert move.sum() > 10
    N = x.shape[0]
    r_det = quadrature.collapsed_gauss(3, (3 * (p - 1)) // 2 + 1)   # degree >= 3(p - 1)
    _, s, _ = oracle.geometry(x, e, 3, p, r_det.xi)
    assert s.min() > 0                                              # no folded element
    rp, ci, M, A, _ = oracle.assemble(x, e, 3, p, r_det.xi, r_det.w)
    assert abs(M.sum() - 1.0) < 1e-13
    Ad = _dense(rp, ci, A, N)
    assert np.abs(Ad.sum(axis=1)).max() < 1e-11
    X = x.T
    assert np.abs(X @ Ad @ X.T - np.eye(3)).max() < 1e-12
    r_mom = quadrature.collapsed_gauss(3, (4 * p - 3) // 2 + 1)    # degree >= 4p - 3
    rp, ci, M, _, _ = oracle.assemble(x, e, 3, p, r_mom.xi, r_mom.w)
    Md = _dense(rp, ci, M, N)
    assert np.abs(X @ Md.sum(axis=1) - 0.5).max() < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4])
def test_tet_lifting_matches_the_node_order(p):
    """Generated order-p tets: every node sits at sum_i (alpha_i / p) x_i of its
    element's corners for the documented multi-index alpha of its local slot;
    the structured cube gets exactly (p n + 1)^3 distinct nodes; interior face
    nodes are shared by exactly two tets."""
    n = 3
    x1, t1 = meshes.kuhn_cube_p2(n, order=1)
    x, e = meshes.to_order(x1, t1, p)
    al = np.array(node_alphas(3, p), float) / p
    pred = np.einsum("ai,eic->eac", al, x[e[:, :4]])
    assert np.abs(x[e] - pred).max() < 1e-15
    assert x.shape[0] == (p * n + 1) ** 3 and len(np.unique(e)) == x.shape[0]
    V = x1.shape[0]
    ne = len(np.unique(np.sort(t1[:, [0, 1, 1, 2, 2, 0, 0, 3, 1, 3, 2, 3]].reshape(-1, 6, 2), axis=2)
                       .reshape(-1, 2), axis=0))
    nfi = (p - 1) * (p - 2) // 2
    if nfi:
        first = V + ne * (p - 1)
        face_nodes = e[:, 4 + 6 * (p - 1):4 + 6 * (p - 1) + 4 * nfi].ravel()
        assert face_nodes.min() == first
        cnt = np.bincount(face_nodes - first)
        assert set(np.unique(cnt)) <= {1, 2}
        on_bnd = np.any((x[first:first + cnt.size] < 1e-12) | (x[first:first + cnt.size] > 1 - 1e-12), axis=1)
        assert np.all(cnt[~on_bnd] == 2) and np.all(cnt[on_bnd] == 1)


def test_tet_face_numbering_is_lexicographic():
    """Face nodes are numbered face by face in lexicographic order of the
    sorted vertex triples (the GPU generator numbers faces the same way)."""
    x1, t1 = meshes.kuhn_cube_p2(2, order=1)
    x, e = meshes.to_order(x1, t1, 3)
    V = x1.shape[0]
    ne = (np.unique(e[:, 4:16]).size) // 2
    first = V + 2 * ne
    faces = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
    tri = np.sort(np.stack([t1[:, list(f)] for f in faces], axis=1), axis=2).reshape(-1, 3)
    uniq = np.unique(tri, axis=0)
    fid = {tuple(t): k for k, t in enumerate(uniq)}
    got = e[:, 16:20].ravel() - first
    assert np.array_equal(got, [fid[tuple(t)] for t in tri])
