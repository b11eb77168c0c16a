"""Seeded synthetic meshes shaped like the paper's workloads (inputs only).

Every generator returns ``(coords, conn)``: coords float64 [N][n] (n = ambient
dimension), conn int32 [nE][ref] with 0-based node indices, corners first
(counter-clockwise), then the edge ("intermediate") nodes, as in the paper's
data-structure convention (Sec. 4.1, Tables elem_array / node_array).

Local edge-node order (0-based):
  segment  : 0, 1 ends, 2 midpoint
  triangle : 3 = (0,1), 4 = (1,2), 5 = (2,0)       (paper's 4:(1,2), 5:(2,3), 6:(3,1))
  tet      : 4 = (0,1), 5 = (1,2), 6 = (2,0), 7 = (0,3), 8 = (1,3), 9 = (2,3)

This module places nodes and builds connectivity; it evaluates no basis
function and computes no element quantity.  Element order is spatially
coherent (children of a refined triangle are consecutive; cubes are visited in
Morton order) and nodes are renumbered by first appearance in the element
list, so that consecutive node ranges are compact patches of the mesh.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "BASE_SEED",
    "icosahedron",
    "icosphere",
    "radial_perturbation",
    "kuhn_cube_p2",
    "boundary_faces_p2",
    "closed_curve_p2",
    "hex_disk",
    "geodesic_sphere",
    "ellipsoid",
    "renumber_first_touch",
    "half_disk_p2",
]

BASE_SEED = 20260514

TRI_EDGES = ((0, 1), (1, 2), (2, 0))
TET_EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))


def icosahedron():
    """The 12 golden-ratio vertices (normalised) and 20 outward-oriented faces."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def _edge_ids(faces: np.ndarray, n_vert: int, local_edges):
    """Unique undirected edges of a simplex list; returns (edges [nEd][2], id [nF][len(local_edges)])."""
    a = np.stack([faces[:, i] for i, _ in local_edges], axis=1)
    b = np.stack([faces[:, j] for _, j in local_edges], axis=1)
    lo = np.minimum(a, b).ravel()
    hi = np.maximum(a, b).ravel()
    key = lo * np.int64(n_vert) + hi
    uniq, inv = np.unique(key, return_inverse=True)
    edges = np.stack([uniq // n_vert, uniq % n_vert], axis=1)
    return edges, inv.reshape(faces.shape[0], len(local_edges))


def renumber_first_touch(coords: np.ndarray, conn: np.ndarray):
    """Renumber nodes in order of first appearance in conn (row-major); unused nodes last."""
    n = coords.shape[0]
    flat = conn.ravel()
    _, first = np.unique(flat, return_index=True)
    used = flat[np.sort(first)]
    order = np.concatenate([used, np.setdiff1d(np.arange(n), used, assume_unique=False)])
    new_id = np.empty(n, dtype=np.int64)
    new_id[order] = np.arange(n)
    return np.ascontiguousarray(coords[order]), new_id[conn].astype(np.int32)


def _subdivide_sphere(level: int):
    v, f = icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        edges, eid = _edge_ids(f, nv, TRI_EDGES)
        mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.vstack([v, mid])
        m01, m12, m20 = (eid[:, k] + nv for k in range(3))
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        # children of (a,b,c) stay consecutive: 4t .. 4t+3, orientation kept.
        ch = np.stack(
            [
                np.stack([a, m01, m20], 1),
                np.stack([m01, b, m12], 1),
                np.stack([m20, m12, c], 1),
                np.stack([m01, m12, m20], 1),
            ],
            axis=1,
        )
        f = ch.reshape(-1, 3)
    return v, f


def _add_p2_edge_nodes(v: np.ndarray, f: np.ndarray, local_edges, project=None):
    nv = v.shape[0]
    edges, eid = _edge_ids(f, nv, local_edges)
    mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
    if project is not None:
        mid = project(mid)
    return np.vstack([v, mid]), np.concatenate([f, eid + nv], axis=1)


def _unit(x):
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def icosphere(level: int, order: int = 1):
    """Unit icosphere: icosahedron refined `level` times, new vertices projected
    to S^2 after each level; for order 2 the final edges' midpoints, projected to
    S^2, become the edge nodes.  Counts: 20*4^level triangles,
    10*4^level + 2 vertices (+ 30*4^level edge nodes for P2)."""
    v, f = _subdivide_sphere(level)
    if order == 2:
        v, f = _add_p2_edge_nodes(v, f, TRI_EDGES, project=_unit)
    elif order != 1:
        raise ValueError(order)
    return renumber_first_touch(v, f)


TET_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))


def _face_alphas(p: int):
    """Interior multi-indices (a_0, a_1, a_2) >= 1 of a triangle, |a| = p, in
    increasing (a_1, a_2)."""
    return [(p - a1 - a2, a1, a2) for a1 in range(1, p) for a2 in range(1, p - a1)]


def to_order(v: np.ndarray, f: np.ndarray, order: int, project=None):
    """Order-p nodes (p = 2, 3, 4) from a P1 curve, triangle or tetrahedron mesh
    (the node generation of the paper's preprocessing, Sec. 4): corners keep
    their numbers; each edge gets p - 1 nodes at lambda = k/p, numbered along
    the edge from its lower to its higher vertex number and shared by the
    elements that meet there.  Triangles then get their (p-1)(p-2)/2 interior
    nodes; tetrahedra get per face the (p-1)(p-2)/2 face nodes, shared by the
    two tets of the face and numbered on the face's vertices sorted by number,
    then per tet its (p-1)(p-2)(p-3)/6 interior nodes.  Node blocks: vertices,
    edge nodes (edges in lexicographic (low, high) order), face nodes (faces in
    lexicographic order of sorted vertex triples), element interior nodes.
    Local order: corners; per local edge (0,1) [, (1,2), (2,0) [, (0,3), (1,3),
    (2,3)]] the nodes from the edge's first corner to its second; triangles:
    interior nodes in increasing (alpha_1, alpha_2); tets: faces (0,1,2),
    (0,1,3), (0,2,3), (1,2,3), each (i, j, l) with its nodes in increasing
    (alpha_j, alpha_l), then interior nodes in increasing (alpha_1, alpha_2,
    alpha_3).  Positions are the straight ones, sum_i lambda_i x_i summed left
    to right (face nodes over the sorted vertices), then `project` if given."""
    if order not in (2, 3, 4):
        raise ValueError(order)
    dim = f.shape[1] - 1
    local_edges = [(0, 1)] if dim == 1 else (TRI_EDGES if dim == 2 else TET_EDGES)
    nv = v.shape[0]
    nE = f.shape[0]
    edges, eid = _edge_ids(f, nv, local_edges)          # edges[k] = (low, high)
    n_e = edges.shape[0]
    cols, pos = [f], [v]
    ts = np.arange(1, order) / order
    # edge nodes along low -> high
    epos = v[edges[:, 0]][:, None, :] * (1 - ts)[None, :, None] + v[edges[:, 1]][:, None, :] * ts[None, :, None]
    pos.append(epos.reshape(-1, v.shape[1]))
    for le, (i, j) in enumerate(local_edges):
        forward = f[:, i] < f[:, j]
        for k in range(1, order):
            kk = np.where(forward, k, order - k)
            cols.append((nv + eid[:, le] * (order - 1) + (kk - 1))[:, None])
    base = nv + n_e * (order - 1)
    if dim == 2:
        alphas = _face_alphas(order)
        n_int = len(alphas)
        ints = []
        for t, al in enumerate(alphas):
            lam = np.array(al, float) / order
            ints.append(lam[0] * v[f[:, 0]] + lam[1] * v[f[:, 1]] + lam[2] * v[f[:, 2]])
            cols.append((base + np.arange(nE) * n_int + t)[:, None])
        if n_int:
            pos.append(np.stack(ints, axis=1).reshape(-1, v.shape[1]))  # element-major numbering
    if dim == 3:
        falphas = _face_alphas(order)
        nfi = len(falphas)
        n_faces = 0
        if nfi:
            tri = np.stack([f[:, list(fc)] for fc in TET_FACES], axis=1)      # [nE][4][3] local vertex order
            srt = np.sort(tri, axis=2).astype(np.int64)
            key = (srt[:, :, 0] * nv + srt[:, :, 1]) * nv + srt[:, :, 2]
            uniq, fid = np.unique(key.ravel(), return_inverse=True)
            fid = fid.reshape(nE, 4)
            n_faces = uniq.shape[0]
            g = np.stack([uniq // (nv * nv), (uniq // nv) % nv, uniq % nv], axis=1)
            fpos = []
            for al in falphas:
                lam = np.array(al, float) / order
                fpos.append(lam[0] * v[g[:, 0]] + lam[1] * v[g[:, 1]] + lam[2] * v[g[:, 2]])
            pos.append(np.stack(fpos, axis=1).reshape(-1, v.shape[1]))
            index = {al: t for t, al in enumerate(falphas)}
            for lf in range(4):
                rank = np.argsort(np.argsort(tri[:, lf, :], axis=1, kind="stable"), axis=1)  # rank of each corner
                for al in falphas:
                    # the node's weights on the sorted vertices, then its number on the face
                    t_of = np.empty(nE, np.int64)
                    for e_al in set(map(tuple, rank)):
                        sel = np.all(rank == np.array(e_al), axis=1)
                        srt_al = [0, 0, 0]
                        for c in range(3):
                            srt_al[e_al[c]] = al[c]
                        t_of[sel] = index[tuple(srt_al)]
                    cols.append((base + fid[:, lf] * nfi + t_of)[:, None])
        cbase = base + n_faces * nfi
        calphas = [(order - a1 - a2 - a3, a1, a2, a3) for a1 in range(1, order) for a2 in range(1, order - a1)
                   for a3 in range(1, order - a1 - a2)]
        n_ci = len(calphas)
        cpos = []
        for t, al in enumerate(calphas):
            lam = np.array(al, float) / order
            cpos.append(lam[0] * v[f[:, 0]] + lam[1] * v[f[:, 1]] + lam[2] * v[f[:, 2]] + lam[3] * v[f[:, 3]])
            cols.append((cbase + np.arange(nE) * n_ci + t)[:, None])
        if n_ci:
            pos.append(np.stack(cpos, axis=1).reshape(-1, v.shape[1]))
    x = np.vstack(pos)
    if project is not None:
        x[nv:] = project(x[nv:])
    conn = np.concatenate(cols, axis=1).astype(np.int32)
    return x, conn


def icosphere_high(level: int, order: int):
    """Unit icosphere with order-3/4 nodes: every generated node projected to S^2."""
    v, f = _subdivide_sphere(level)
    return to_order(v, f, order, project=_unit)


def radial_perturbation(coords: np.ndarray, amp: float = 0.2):
    """Map every node radially to r(theta, phi) = 1 + amp sin(3 theta) cos(2 phi)
    (theta polar angle from +z, phi = atan2(y, x)); nodes assumed on S^2 first."""
    u = _unit(coords)
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    r = 1.0 + amp * np.sin(3.0 * theta) * np.cos(2.0 * phi)
    return u * r[:, None]


def ellipsoid(level: int, axes=(1.0, 0.8, 0.6), sigma: float = 1e-3, seed: int = BASE_SEED + 5):
    """P2 icosphere scaled to semi-axes `axes` plus seeded N(0, sigma^2) noise per coordinate."""
    x, e = icosphere(level, 2)
    x = x * np.asarray(axes)[None, :]
    if sigma > 0:
        rng = np.random.default_rng(seed)
        x = x + rng.normal(0.0, sigma, size=x.shape)
    return np.ascontiguousarray(x), e


def _morton3(i, j, k, bits):
    code = np.zeros_like(i, dtype=np.int64)
    for b in range(bits):
        code |= ((i >> b) & 1) << (3 * b + 2)
        code |= ((j >> b) & 1) << (3 * b + 1)
        code |= ((k >> b) & 1) << (3 * b)
    return code


def kuhn_cube_p2(n: int = 64, jitter: float = 0.1, seed: int = BASE_SEED + 3, order: int = 2):
    """Unit cube, n^3 cells, each Kuhn-split into 6 tetrahedra along the 6 axis
    permutations from the cell's min corner.  Each vertex coordinate component is
    jittered by U(-jitter*h, jitter*h) unless the vertex lies on a boundary plane
    normal to that axis (keeps the cube exact).  P2 edge nodes at straight
    midpoints (affine tets).  Tets are oriented positively; cells in Morton order."""
    h = 1.0 / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    vid = (I * (n + 1) + J) * (n + 1) + K
    x = np.stack([I, J, K], axis=-1).reshape(-1, 3).astype(np.float64) * h
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter * h, jitter * h, size=x.shape)
    idx = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    on_bnd = (idx == 0) | (idx == n)
    x = x + np.where(on_bnd, 0.0, jit)

    c = np.arange(n)
    ci, cj, ck = [a.ravel() for a in np.meshgrid(c, c, c, indexing="ij")]
    bits = max(1, int(np.ceil(np.log2(max(n, 2)))))
    order_cells = np.argsort(_morton3(ci, cj, ck, bits), kind="stable")
    ci, cj, ck = ci[order_cells], cj[order_cells], ck[order_cells]
    perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for p in perms:
        s1 = unit[p[0]]
        s2 = s1 + unit[p[1]]
        s3 = s2 + unit[p[2]]
        verts = []
        for s in (np.zeros(3, np.int64), s1, s2, s3):
            verts.append(vid[ci + s[0], cj + s[1], ck + s[2]])
        tets.append(np.stack(verts, axis=1))
    t = np.stack(tets, axis=1).reshape(-1, 4)  # 6 consecutive tets per cell
    # positive orientation
    d = x[t[:, 1:]] - x[t[:, :1]]
    neg = np.linalg.det(d) < 0
    t[neg] = t[neg][:, [0, 2, 1, 3]]
    if order == 2:
        x, t = _add_p2_edge_nodes(x, t, TET_EDGES)
    return renumber_first_touch(x, t)


def boundary_faces_p2(conn_tet: np.ndarray):
    """Boundary triangles of a P2 tet mesh (faces used once), as P2 triangles in
    the bulk node numbering: corners then edge nodes (0,1), (1,2), (2,0)."""
    # local faces (corner triples) of a tet and, per face edge, the tet edge-node slot.
    faces = ((0, 2, 1), (0, 1, 3), (1, 2, 3), (0, 3, 2))
    edge_slot = {}
    for s, (i, j) in enumerate(TET_EDGES):
        edge_slot[(i, j)] = 4 + s
        edge_slot[(j, i)] = 4 + s
    tris = []
    for fc in faces:
        cols = list(fc) + [edge_slot[(fc[0], fc[1])], edge_slot[(fc[1], fc[2])], edge_slot[(fc[2], fc[0])]]
        tris.append(conn_tet[:, cols])
    tri = np.stack(tris, axis=1).reshape(-1, 6)
    key = np.sort(tri[:, :3], axis=1).astype(np.int64)
    nmax = int(conn_tet.max()) + 1
    k = (key[:, 0] * nmax + key[:, 1]) * nmax + key[:, 2]
    _, inv, cnt = np.unique(k, return_inverse=True, return_counts=True)
    once = cnt[inv] == 1
    return np.ascontiguousarray(tri[once].astype(np.int32))


def closed_curve_p2(n_seg: int, seed: int, n_modes: int = 8):
    """Closed star-shaped P2 curve in R^2: r(phi) = 1 + sum_m a_m cos(m phi + beta_m),
    a_m ~ U(0, 0.3/m), beta_m ~ U(0, 2 pi); nodes at equal phi (ends, then midpoints)."""
    rng = np.random.default_rng(seed)
    m = np.arange(1, n_modes + 1)
    a = rng.uniform(0.0, 0.3 / m)
    beta = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    phi = np.arange(2 * n_seg) * (np.pi / n_seg)  # vertices at even k, midpoints at odd k
    r = 1.0 + (a[None, :] * np.cos(m[None, :] * phi[:, None] + beta[None, :])).sum(axis=1)
    pts = np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)
    k = np.arange(n_seg)
    conn = np.stack([2 * k, (2 * k + 2) % (2 * n_seg), 2 * k + 1], axis=1)
    return renumber_first_touch(pts, conn)


def _grid_triangles(f: int):
    """Barycentric grid of a triangle at frequency f: integer (i, j) points with
    i + j <= f and the f^2 small triangles (counter-clockwise) as index triples."""
    pts = [(i, j) for i in range(f + 1) for j in range(f + 1 - i)]
    index = {p: k for k, p in enumerate(pts)}
    tris = []
    for i in range(f):
        for j in range(f - i):
            tris.append((index[(i, j)], index[(i + 1, j)], index[(i, j + 1)]))
            if i + j < f - 1:
                tris.append((index[(i + 1, j)], index[(i + 1, j + 1)], index[(i, j + 1)]))
    return np.array(pts, dtype=np.int64), np.array(tris, dtype=np.int64)


def _subdivide_faces(corners: np.ndarray, faces: np.ndarray, f: int):
    """Class-I subdivision of every face at frequency f with shared nodes on
    shared edges/corners (keys are exact integer lattice points of each face,
    canonicalised through the global corner ids)."""
    gp, gt = _grid_triangles(f)
    nf = faces.shape[0]
    # point (i, j) of face (A, B, C): A + i/f (B - A) + j/f (C - A); barycentric (f-i-j, i, j)
    bary = np.stack([f - gp[:, 0] - gp[:, 1], gp[:, 0], gp[:, 1]], axis=1)  # [P][3]
    # canonical key: sorted (corner id, weight) pairs; a point on an edge / corner
    # gets the same key from every face that contains it.
    ids = faces[:, None, :].repeat(gp.shape[0], axis=1)  # [nf][P][3]
    w = np.broadcast_to(bary[None], ids.shape)
    ids_m = np.where(w > 0, ids, -1)
    o = np.argsort(ids_m, axis=2)
    ids_s = np.take_along_axis(ids_m, o, 2)
    w_s = np.take_along_axis(w, o, 2)
    nc = corners.shape[0] + 1
    key = np.zeros(ids_s.shape[:2], dtype=np.int64)
    for k in range(3):
        key = key * nc + (ids_s[:, :, k] + 1)
        key = key * (f + 1) + w_s[:, :, k]
    uniq, first, inv = np.unique(key.ravel(), return_index=True, return_inverse=True)
    inv = inv.reshape(nf, -1)
    fi = first // gp.shape[0]
    pi = first % gp.shape[0]
    A, B, C = (corners[faces[fi, k]] for k in range(3))
    bw = bary[pi].astype(np.float64) / f
    pts = bw[:, :1] * A + bw[:, 1:2] * B + bw[:, 2:3] * C
    tri = inv[:, gt].reshape(-1, 3)
    return pts, tri


def geodesic_sphere(f: int, order: int = 2, amp: float = 0.2):
    """Class-I geodesic icosphere at frequency f (20 f^2 triangles), projected to
    S^2, P2 edge nodes at projected chord midpoints, then radially perturbed."""
    v, fc = icosahedron()
    pts, tri = _subdivide_faces(v, fc, f)
    pts = _unit(pts)
    if order == 2:
        pts, tri = _add_p2_edge_nodes(pts, tri, TRI_EDGES, project=_unit)
    pts = radial_perturbation(pts, amp) if amp else pts
    return renumber_first_touch(pts, tri)


def hex_disk(f: int, order: int = 2):
    """Planar unit disk: regular hexagon (6 triangles around the centre),
    subdivided at frequency f (6 f^2 triangles), every node mapped radially
    p -> p / |p| * hexnorm(p) so the hexagon boundary lands on the unit circle."""
    ang = np.arange(6) * (np.pi / 3)
    corners = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1)])
    faces = np.array([[0, 1 + k, 1 + (k + 1) % 6] for k in range(6)], dtype=np.int64)
    pts, tri = _subdivide_faces(corners, faces, f)
    if order == 2:
        pts, tri = _add_p2_edge_nodes(pts, tri, TRI_EDGES)

    r = np.linalg.norm(pts, axis=1)
    # hexagon "norm": max over the 6 edge normals of <p, n_k> / apothem
    nrm_ang = ang + np.pi / 6
    normals = np.stack([np.cos(nrm_ang), np.sin(nrm_ang)], 1)
    apothem = np.cos(np.pi / 6)
    hn = (pts @ normals.T).max(axis=1) / apothem
    scale = np.where(r > 0, hn / np.where(r > 0, r, 1.0), 0.0)
    pts = pts * scale[:, None]
    return renumber_first_touch(pts, tri)


def half_disk_p2():
    """The paper's worked P2 half-disk mesh (Sec. 4.1, Tables elem_array and
    node_array), 0-based.  The printed nodes 6 and 9 ("-sqrt2, sqrt2" twice) are
    read as (-sqrt(2)/2, sqrt(2)/2) and (sqrt(2)/2, sqrt(2)/2), the points of the
    unit half circle between nodes 1-3 and 3-7 that the figure draws."""
    s = 0.5 * 2.0 ** 0.5
    coords = np.array(
        [[-1, 0], [0, 0], [0, 1], [-0.5, 0], [0, 0.5], [-s, s], [1, 0], [0.5, 0], [s, s]], dtype=np.float64
    )
    conn = np.array([[1, 2, 3, 4, 5, 6], [2, 7, 3, 8, 9, 5]], dtype=np.int32) - 1
    return coords, conn


def batch_item(i: int, n_meshes: int = 512, scale: float = 1.0, seed: int = BASE_SEED + 4):
    """Mesh i of the uneven batch: family i mod 3 = closed P2 curve
    (1k..200k segments), planar hexagonal disk (5k..500k triangles, P1 and P2
    alternating), P2 perturbed geodesic sphere (20k..1.31M triangles); sizes
    log-uniform, drawn from a generator seeded by (seed, i) so every item can be
    built on its own; `scale` shrinks every size.  Returns
    (family, coords, conn, dim, order)."""
    del n_meshes
    rng = np.random.default_rng([seed, i])
    u = rng.random()
    fam = i % 3
    if fam == 0:
        n = int(round(np.exp(np.log(1e3) + u * (np.log(2e5) - np.log(1e3))) * scale))
        x, e = closed_curve_p2(max(n, 8), seed=seed * 1000 + i)
        return "curve_p2", x, e, 1, 2
    if fam == 1:
        t = np.exp(np.log(5e3) + u * (np.log(5e5) - np.log(5e3))) * scale
        f = max(2, int(round((t / 6.0) ** 0.5)))
        order = 2 if (i // 3) % 2 == 0 else 1
        x, e = hex_disk(f, order)
        return f"disk_p{order}", x, e, 2, order
    t = np.exp(np.log(2e4) + u * (np.log(1.31e6) - np.log(2e4))) * scale
    f = max(2, int(round((t / 20.0) ** 0.5)))
    x, e = geodesic_sphere(f, 2)
    return "sphere_p2", x, e, 2, 2


def batch_workload(n_meshes: int = 512, scale: float = 1.0, seed: int = BASE_SEED + 4):
    """The whole uneven batch (see batch_item)."""
    return [batch_item(i, n_meshes, scale, seed) for i in range(n_meshes)]
