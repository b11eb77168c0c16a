"""Order-p node generation from an order-1 mesh -- test infrastructure only.

Only the tests may call this.  It restates, with plain loops and no shared
code, the node generation of the paper's preprocessing (Sec. 4: the nodes of
an order-p element at alpha / p in barycentric coordinates) under the library's
documented numbering:

  * the P1 vertices keep their numbers;
  * then p - 1 nodes per edge, edges in lexicographic order of their
    (low, high) vertex numbers, each edge's nodes from its low to its high
    vertex at x_lo (1 - k/p) + x_hi (k/p);
  * triangles: then each element's interior nodes (element by element), in
    increasing (alpha_1, alpha_2), at sum_i (alpha_i / p) x_i;
  * tetrahedra: then the nodes of every face -- faces in lexicographic order of
    their sorted vertex triples (g0 < g1 < g2), each face's nodes by increasing
    (a_1, a_2) at (a_0/p) x_g0 + (a_1/p) x_g1 + (a_2/p) x_g2 -- then each
    tet's interior nodes in increasing (alpha_1, alpha_2, alpha_3).

Local order of an element's nodes: corners; per local edge (0,1) [, (1,2),
(2,0) [, (0,3), (1,3), (2,3)]] its nodes from the edge's first corner to its
second; then (triangles) the interior nodes in increasing (alpha_1, alpha_2);
(tetrahedra) the faces (0,1,2), (0,1,3), (0,2,3), (1,2,3), each face (i, j, l)
with its nodes in increasing (alpha_j, alpha_l), then the interior nodes.
Every position is evaluated as products, then sums left to right.
"""
from __future__ import annotations

import numpy as np

_EDGES = {1: [(0, 1)], 2: [(0, 1), (1, 2), (2, 0)], 3: [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]}
_TET_FACES = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


def _tri_alphas(p):
    """(a_0, a_1, a_2) with every entry >= 1 and sum p, in increasing (a_1, a_2)."""
    out = []
    for a1 in range(1, p):
        for a2 in range(1, p - a1):
            out.append((p - a1 - a2, a1, a2))
    return out


def _tet_alphas(p):
    """(a_0, .., a_3) with every entry >= 1 and sum p, in increasing (a_1, a_2, a_3)."""
    out = []
    for a1 in range(1, p):
        for a2 in range(1, p - a1):
            for a3 in range(1, p - a1 - a2):
                out.append((p - a1 - a2 - a3, a1, a2, a3))
    return out


def _combo(weights, points):
    """sum_i weights[i] * points[i], products first, then summed left to right."""
    acc = weights[0] * points[0]
    for w, x in zip(weights[1:], points[1:]):
        acc = acc + w * x
    return acc


def lift_order(v, f, order):
    """Order-p nodes (p = 2, 3, 4) of the order-1 curve, triangle or
    tetrahedron mesh (v, f).  Returns (coords [n][ambient], conn [nE][ref])."""
    v = np.asarray(v, dtype=np.float64)
    f = np.asarray(f, dtype=np.int64)
    p = int(order)
    if p not in (2, 3, 4):
        raise ValueError(order)
    dim = f.shape[1] - 1
    nv, nE = v.shape[0], f.shape[0]
    edges = sorted({(min(f[e, i], f[e, j]), max(f[e, i], f[e, j])) for e in range(nE) for i, j in _EDGES[dim]})
    edge_id = {ed: k for k, ed in enumerate(edges)}
    pos = [v[i] for i in range(nv)]
    for lo, hi in edges:
        for k in range(1, p):
            t = k / p
            pos.append(v[lo] * (1.0 - t) + v[hi] * t)
    base = nv + len(edges) * (p - 1)
    falphas = _tri_alphas(p)
    faces, face_id = [], {}
    if dim == 3:
        faces = sorted({tuple(sorted(int(f[e, c]) for c in fc)) for e in range(nE) for fc in _TET_FACES})
        face_id = {fc: k for k, fc in enumerate(faces)}
        for g in faces:
            for al in falphas:
                pos.append(_combo([a / p for a in al], [v[g[0]], v[g[1]], v[g[2]]]))
        ibase = base + len(faces) * len(falphas)
        ialphas = _tet_alphas(p)
    else:
        ibase = base
        ialphas = falphas if dim == 2 else []
    for e in range(nE):
        for al in ialphas:
            pos.append(_combo([a / p for a in al], [v[f[e, c]] for c in range(dim + 1)]))
    conn = []
    for e in range(nE):
        row = [int(f[e, c]) for c in range(dim + 1)]
        for i, j in _EDGES[dim]:
            k_e = edge_id[(min(f[e, i], f[e, j]), max(f[e, i], f[e, j]))]
            for k in range(1, p):
                kk = k if f[e, i] < f[e, j] else p - k
                row.append(nv + k_e * (p - 1) + kk - 1)
        if dim == 3:
            for fc in _TET_FACES:
                g = tuple(sorted(int(f[e, c]) for c in fc))
                for _, aj, al in _tri_alphas(p):
                    local = {int(f[e, fc[0]]): p - aj - al, int(f[e, fc[1]]): aj, int(f[e, fc[2]]): al}
                    s = (local[g[0]], local[g[1]], local[g[2]])
                    row.append(base + face_id[g] * len(falphas) + falphas.index(s))
        row.extend(ibase + e * len(ialphas) + t for t in range(len(ialphas)))
        conn.append(row)
    return np.array(pos, dtype=np.float64).reshape(len(pos), v.shape[1]), np.array(conn, dtype=np.int32)
