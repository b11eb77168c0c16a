"""Seeded parity cases: one small mesh per supported (dim, ambient, order),
sized so the oracle finishes in well under a second but the pattern spans
several row tiles (tests retile to the minimum capacity) with a ragged tail."""
from __future__ import annotations

import numpy as np

from paper_2605_14035_gb300.inputs import meshes, quadrature


def coef_field(pts: np.ndarray) -> np.ndarray:
    """c = 1 + x^2 + y z at physical quadrature points (missing coordinates read as 0.5)."""
    x = pts[..., 0]
    y = pts[..., 1] if pts.shape[-1] > 1 else 0.5
    z = pts[..., 2] if pts.shape[-1] > 2 else 0.5
    return 1.0 + x * x + y * z


def _curve_p1(n, seed):
    x, e = meshes.closed_curve_p2(n, seed)
    # vertices are the nodes shared by two segments; keep the P1 segments (ends only)
    conn = e[:, :2].copy()
    used = np.unique(conn)
    new = -np.ones(x.shape[0], dtype=np.int64)
    new[used] = np.arange(used.size)
    return np.ascontiguousarray(x[used]), new[conn].astype(np.int32)


def _space_curve_p2(n, seed):
    x, e = meshes.closed_curve_p2(n, seed)
    phi = np.arctan2(x[:, 1], x[:, 0])
    z = 0.2 * np.sin(3 * phi)
    return np.ascontiguousarray(np.column_stack([x, z])), e


def _interval_p2(n):
    # [0, 1] with graded nodes; P2: ends then midpoint
    t = np.linspace(0, 1, n + 1) ** 1.3
    mids = 0.5 * (t[:-1] + t[1:])
    x = np.concatenate([t, mids])[:, None]
    k = np.arange(n)
    return x, np.stack([k, k + 1, n + 1 + k], 1).astype(np.int32)


def build_cases():
    """name -> (coords, conn, dim, order, rule)."""
    c = {}
    r_tri3, r_tri7 = quadrature.tri_3pt_deg2(), quadrature.tri_7pt_deg5()
    r_tet14, r_tet4 = quadrature.tet_14pt_deg5(), quadrature.tet_4pt_deg2()
    r_g3 = quadrature.gauss_interval(3)
    c["sphere_p1"] = (*meshes.icosphere(3, 1), 2, 1, r_tri3)
    c["ellipsoid_p2"] = (*meshes.ellipsoid(2, sigma=1e-2, seed=3), 2, 2, r_tri7)
    x, e = meshes.icosphere(3, 2)
    c["perturbed_sphere_p2"] = (meshes.radial_perturbation(x), e, 2, 2, r_tri7)
    c["disk_p1"] = (*meshes.hex_disk(7, 1), 2, 1, r_tri3)
    c["disk_p2"] = (*meshes.hex_disk(5, 2), 2, 2, r_tri7)
    c["half_disk_p2"] = (*meshes.half_disk_p2(), 2, 2, r_tri7)
    c["curve_p2"] = (*meshes.closed_curve_p2(400, seed=9), 1, 2, r_g3)
    c["curve_p1"] = (*_curve_p1(300, 4), 1, 1, quadrature.gauss_interval(2))
    c["space_curve_p2"] = (*_space_curve_p2(250, 5), 1, 2, r_g3)
    c["interval_p2"] = (*_interval_p2(200), 1, 2, r_g3)
    c["cube_p2"] = (*meshes.kuhn_cube_p2(4), 3, 2, r_tet14)
    c["cube_p1"] = (*meshes.kuhn_cube_p2(5, order=1), 3, 1, r_tet4)
    xc, ec = meshes.kuhn_cube_p2(3)
    c["cube_boundary_p2"] = (xc, meshes.boundary_faces_p2(ec), 2, 2, r_tri7)  # rows of interior nodes empty
    # rules other than the compile-time ones take the general (lane-pair) path
    x, e = meshes.icosphere(2, 2)
    c["sphere_p2_gauss9"] = (meshes.radial_perturbation(x), e, 2, 2, quadrature.collapsed_gauss(2, 3))
    c["disk_p1_gauss4"] = (*meshes.hex_disk(8, 1), 2, 1, quadrature.collapsed_gauss(2, 2))
    c["cube_p2_gauss8"] = (*meshes.kuhn_cube_p2(3), 3, 2, quadrature.collapsed_gauss(3, 2))
    # the rule sizes the paper uses for P2 (order 10 / 8 / 7 in 1-D / 2-D / 3-D)
    c["ellipsoid_p2_paper16"] = (*meshes.ellipsoid(2, sigma=1e-2, seed=6), 2, 2, quadrature.paper_rule(2))
    c["curve_p2_paper6"] = (*meshes.closed_curve_p2(120, seed=10), 1, 2, quadrature.paper_rule(1))
    c["cube_p2_paper64"] = (*meshes.kuhn_cube_p2(2), 3, 2, quadrature.paper_rule(3))
    # orders 3 and 4 (curves and triangles): element-major path, general Jacobian
    r16 = quadrature.tri_16pt_deg8()
    c["sphere_p3"] = (*meshes.icosphere_high(1, 3), 2, 3, r16)
    c["sphere_p4"] = (*meshes.icosphere_high(1, 4), 2, 4, r16)
    xd, ed = meshes.hex_disk(4, 1)
    c["disk_p3"] = (*meshes.to_order(xd, ed, 3), 2, 3, r16)
    t = 2 * np.pi * np.arange(40) / 40
    xc = np.stack([np.cos(t), np.sin(t)], axis=1)
    ec = np.stack([np.arange(40), (np.arange(40) + 1) % 40], axis=1).astype(np.int32)
    unit = lambda y: y / np.linalg.norm(y, axis=1, keepdims=True)  # noqa: E731
    c["circle_p4"] = (*meshes.to_order(xc, ec, 4, project=unit), 1, 4, quadrature.gauss_interval(6))
    # orders 3 and 4 on tetrahedra (warp-per-element path): curved elements
    c["cube_p3"] = (*curved_cube(3, 3), 3, 3, quadrature.paper_rule(3))
    c["cube_p4"] = (*curved_cube(2, 4), 3, 4, quadrature.paper_rule(3))
    c["cube_p3_gauss27"] = (*curved_cube(2, 3, seed=13), 3, 3, quadrature.collapsed_gauss(3, 3))
    return c


def curved_cube(n, order, amp=0.004, seed=12):
    """Order-p Kuhn cube (n^3 cells) whose generated interior nodes are moved by
    U(-amp, amp) per component: curved edges, faces and cells, flat boundary."""
    x1, t1 = meshes.kuhn_cube_p2(n, order=1)
    x, e = meshes.to_order(x1, t1, order)
    on_bnd = np.any((x < 1e-12) | (x > 1 - 1e-12), axis=1)
    move = ~on_bnd & (np.arange(x.shape[0]) >= x1.shape[0])
    rng = np.random.default_rng(meshes.BASE_SEED + seed)
    return x + np.where(move[:, None], rng.uniform(-amp, amp, x.shape), 0.0), e


def diag_scaled_error(v, ref, rp, ci):
    """max_ij |v_ij - ref_ij| / sqrt(|ref_ii| |ref_jj|) (0/0 counts as 0)."""
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    diag = np.zeros(n)
    is_d = rows == ci
    diag[rows[is_d]] = np.abs(ref[is_d])
    den = np.sqrt(diag[rows] * diag[ci])
    num = np.abs(v - ref)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(num == 0, 0.0, num / den)
    return float(np.max(r)) if r.size else 0.0
