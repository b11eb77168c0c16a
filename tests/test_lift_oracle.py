"""The oracle's order-p node generation (oracle.lift_order), pinned to the
definition it restates: every node of every element sits at sum_i (alpha_i/p)
x_i of the element's corners for the multi-index alpha of its local slot in
the documented order; distinct numbers are distinct points and each point has
one number; the closed sphere has V + (p-1) E + (p-1)(p-2)/2 F nodes and the
structured cube (p n + 1)^3.  The input generator's vectorised version gives
the same bits (two independent restatements agree)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2605_14035_gb300.inputs import meshes


def local_alphas(dim, p):
    """Multi-indices (over the corners) of the local nodes, in the documented order."""
    corners = [tuple(p if c == k else 0 for c in range(dim + 1)) for k in range(dim + 1)]
    edges = {1: [(0, 1)], 2: [(0, 1), (1, 2), (2, 0)], 3: [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]}[dim]
    out = list(corners)
    for i, j in edges:
        for k in range(1, p):
            a = [0] * (dim + 1)
            a[i], a[j] = p - k, k
            out.append(tuple(a))
    inner = [(a1, a2) for a1 in range(1, p) for a2 in range(1, p - a1)]
    if dim == 2:
        out += [(p - a1 - a2, a1, a2) for a1, a2 in inner]
    if dim == 3:
        for fi, fj, fl in [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]:
            for aj, al in inner:
                a = [0] * 4
                a[fi], a[fj], a[fl] = p - aj - al, aj, al
                out.append(tuple(a))
        out += [(p - a1 - a2 - a3, a1, a2, a3) for a1 in range(1, p) for a2 in range(1, p - a1)
                for a3 in range(1, p - a1 - a2)]
    return np.array(out, float) / p


def _circle(n):
    t = 2 * np.pi * np.arange(n) / n
    return (np.stack([np.cos(t), np.sin(t)], 1),
            np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32))


MESHES = {
    "circle": lambda: _circle(17),
    "sphere": lambda: meshes.icosphere(1, 1),
    "disk": lambda: meshes.hex_disk(3, 1),
    "cube": lambda: meshes.kuhn_cube_p2(2, order=1),
    "cube_jit": lambda: meshes.kuhn_cube_p2(2, jitter=0.2, seed=meshes.BASE_SEED + 21, order=1),
}


@pytest.mark.parametrize("name,p", list(itertools.product(MESHES, (2, 3, 4))))
def test_lift_order_nodes_at_documented_positions(name, p):
    v, f = MESHES[name]()
    dim = f.shape[1] - 1
    x, e = oracle.lift_order(v, f, p)
    al = local_alphas(dim, p)
    assert e.shape[1] == al.shape[0]
    assert np.array_equal(e[:, :dim + 1], f)
    pred = np.einsum("ai,eic->eac", al, v[f])
    assert np.abs(x[e] - pred).max() < 1e-15
    # numbers <-> points one to one, every generated number used
    assert len(np.unique(e)) == x.shape[0]
    key = np.round(x / 1e-9).astype(np.int64)
    assert len(np.unique(key, axis=0)) == x.shape[0]
    if name == "sphere":
        F = f.shape[0]
        V, E = F // 2 + 2, 3 * F // 2
        assert x.shape[0] == V + (p - 1) * E + (p - 1) * (p - 2) // 2 * F
    if name == "cube":
        assert x.shape[0] == (p * 2 + 1) ** 3


@pytest.mark.parametrize("name,p", list(itertools.product(MESHES, (2, 3, 4))))
def test_lift_order_matches_the_input_generator(name, p):
    v, f = MESHES[name]()
    xo, eo = oracle.lift_order(v, f, p)
    xg, eg = meshes.to_order(v, f, p)
    assert np.array_equal(eo, eg)
    assert np.array_equal(xo.view(np.int64), xg.view(np.int64))
