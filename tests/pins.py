"""Checks that pin the oracle to facts outside itself.

Each check returns an error measure; the tests assert it is below a bound,
and the planted-mistake tests assert that at least one check fails for every
planted mistake.  Nothing here comes from the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import oracle
from exact import affine_nodes, exact_mass_ref, exact_stiffness, simplex_measure
from paper_2605_14035_gb300.inputs import meshes, quadrature

RNG = np.random.default_rng(12345)

# Reference nodes of the simplices in the documented local order (orders 3, 4 added below).
REF_NODES = {
    (1, 1): np.array([[0.0], [1.0]]),
    (1, 2): np.array([[0.0], [1.0], [0.5]]),
    (2, 1): np.array([[0, 0], [1, 0], [0, 1]], float),
    (2, 2): np.array([[0, 0], [1, 0], [0, 1], [0.5, 0], [0.5, 0.5], [0, 0.5]], float),
    (3, 1): np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
    (3, 2): np.array(
        [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.5, 0, 0], [0.5, 0.5, 0], [0, 0.5, 0],
         [0, 0, 0.5], [0.5, 0, 0.5], [0, 0.5, 0.5]], float),
}


def _high_order_nodes(d, p):
    """Reference coordinates of the order-p nodes (p = 3, 4) in the documented
    order: corners; per edge ((0,1); (0,1),(1,2),(2,0); those and (0,3),(1,3),
    (2,3)) the nodes ((p-k) e_i + k e_j)/p; triangles: interior by increasing
    (a1, a2); tets: faces (0,1,2),(0,1,3),(0,2,3),(1,2,3), each (i,j,l) by
    increasing (a_j, a_l), then the interior by increasing (a1, a2, a3)."""
    al = [[p if c == i else 0 for c in range(d + 1)] for i in range(d + 1)]
    edges = {1: [(0, 1)], 2: [(0, 1), (1, 2), (2, 0)], 3: [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]}[d]
    for i, j in edges:
        for k in range(1, p):
            a = [0] * (d + 1)
            a[i], a[j] = p - k, k
            al.append(a)
    if d == 2:
        al += [[p - a1 - a2, a1, a2] for a1 in range(1, p) for a2 in range(1, p - a1)]
    if d == 3:
        for i, j, l in [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]:
            for aj in range(1, p):
                for a_l in range(1, p - aj):
                    a = [0] * 4
                    a[i], a[j], a[l] = p - aj - a_l, aj, a_l
                    al.append(a)
        al += [[p - a1 - a2 - a3, a1, a2, a3] for a1 in range(1, p) for a2 in range(1, p - a1)
               for a3 in range(1, p - a1 - a2)]
    return np.array(al, float)[:, 1:] / p


for _d in (1, 2, 3):
    for _p in (3, 4):
        REF_NODES[(_d, _p)] = _high_order_nodes(_d, _p)

COMBOS = [(1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]  # (d, n)


def csr(vals, pat, n):
    return sp.csr_matrix((vals, pat[1], pat[0]), shape=(n, n))


def check_lagrange(mutation=0):
    """phi_a(node_b) = delta_ab (Eq. F_map's Lagrange property) and sum phi = 1."""
    err = 0.0
    for (d, p), nodes in REF_NODES.items():
        phi, dphi = oracle.tabulate(d, p, nodes, mutation)
        err = max(err, np.abs(phi - np.eye(len(nodes))).max())
        pts = RNG.dirichlet(np.ones(d + 1), size=5)[:, 1:]
        phi2, dphi2 = oracle.tabulate(d, p, pts, mutation)
        err = max(err, np.abs(phi2.sum(1) - 1).max(), np.abs(dphi2.sum(1)).max())
        # gradients against central differences of the values
        h = 1e-6
        for m in range(d):
            e = np.zeros(d)
            e[m] = h
            fp, _ = oracle.tabulate(d, p, pts + e, mutation)
            fm, _ = oracle.tabulate(d, p, pts - e, mutation)
            err = max(err, np.abs((fp - fm) / (2 * h) - dphi2[:, :, m]).max() * 1e-3)
    return err


def random_simplex(d, n, rng=RNG):
    """A well-shaped random simplex in R^n (d <= n)."""
    while True:
        v = rng.normal(size=(d + 1, n))
        E = (v[1:] - v[0]).T
        G = E.T @ E
        if np.linalg.cond(G) < 20:
            return v


def check_affine_exact(mutation=0):
    """Single affine elements against exact rationals x |T| (mass) and the
    barycentric-gradient formula (stiffness), for every (d, n, p)."""
    err = 0.0
    for d, n in COMBOS:
        for p in (1, 2):
            v = random_simplex(d, n)
            x = affine_nodes(v, p)
            conn = np.arange(len(x), dtype=np.int32)[None, :]
            rule = quadrature.default_rule(d, 2)  # degree >= 2p exact for affine mass
            M, A, _ = oracle.local_matrices(x, conn, d, p, rule.xi, rule.w, mutation=mutation)
            T = simplex_measure(v)
            Mex = np.array(exact_mass_ref(d, p), dtype=float) * T
            Aex = exact_stiffness(v, p)
            err = max(err, np.abs(M[0] - Mex).max() / np.abs(Mex).max(), np.abs(A[0] - Aex).max() / np.abs(Aex).max())
    return err


def cross2(a, b):
    return a[0] * b[1] - a[1] * b[0]


def check_p1_closed_forms(mutation=0):
    """P1 triangle |T|/12 [2 1 1; 1 2 1; 1 1 2]; tet |T|/20 (1 + delta); interval
    h/6 [2 1; 1 2]; triangle stiffness = cotangent formula."""
    err = 0.0
    v = np.array([[0.1, 0.2], [1.3, 0.1], [0.4, 0.9]])
    conn = np.arange(3, dtype=np.int32)[None]
    r = quadrature.tri_3pt_deg2()
    M, A, _ = oracle.local_matrices(v, conn, 2, 1, r.xi, r.w, mutation=mutation)
    T = 0.5 * abs(cross2(v[1] - v[0], v[2] - v[0]))
    err = max(err, np.abs(M[0] - T / 12 * (np.ones((3, 3)) + np.eye(3))).max() / T)
    cot = np.zeros(3)
    for k in range(3):
        a, b = v[(k + 1) % 3] - v[k], v[(k + 2) % 3] - v[k]
        cot[k] = np.dot(a, b) / abs(cross2(a, b))
    Acot = np.zeros((3, 3))
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        Acot[i, j] = Acot[j, i] = -0.5 * cot[k]
    Acot[np.diag_indices(3)] = -Acot.sum(1)
    err = max(err, np.abs(A[0] - Acot).max())
    vt = random_simplex(3, 3)
    r3 = quadrature.tet_4pt_deg2()
    M, _, _ = oracle.local_matrices(vt, np.arange(4, dtype=np.int32)[None], 3, 1, r3.xi, r3.w, mutation=mutation)
    Tt = abs(np.linalg.det(vt[1:] - vt[0])) / 6
    err = max(err, np.abs(M[0] - Tt / 20 * (np.ones((4, 4)) + np.eye(4))).max() / Tt)
    vs = np.array([[0.3, -0.2], [1.0, 0.4]])
    r1 = quadrature.gauss_interval(2)
    M, _, _ = oracle.local_matrices(vs, np.arange(2, dtype=np.int32)[None], 1, 1, r1.xi, r1.w, mutation=mutation)
    h = np.linalg.norm(vs[1] - vs[0])
    err = max(err, np.abs(M[0] - h / 6 * np.array([[2, 1], [1, 2]])).max() / h)
    return err


def half_disk_area(mutation=0):
    x, e = meshes.half_disk_p2()
    r = quadrature.tri_7pt_deg5()
    _, _, M, A, _ = oracle.assemble(x, e, 2, 2, r.xi, r.w, mutation=mutation)
    return M.sum()


def check_half_disk(mutation=0):
    """Worked mesh of Sec. 4.1: exact area 1 + (4/3)(sqrt2 - 1) (det J is quadratic,
    integrated exactly by the degree-5 rule); A.1 = 0."""
    exact = 1.0 + 4.0 / 3.0 * (2.0 ** 0.5 - 1.0)
    return abs(half_disk_area(mutation) - exact) / exact


def check_sphere_invariants(level=2, order=2, mutation=0):
    """A.1 = 0 (partition of unity), symmetry, and 1^T M 1 close to 4 pi."""
    x, e = meshes.icosphere(level, order)
    r = quadrature.default_rule(2, order)
    pat = oracle.pattern(e, x.shape[0])
    _, _, M, A, _ = oracle.assemble(x, e, 2, order, r.xi, r.w, pat=pat, mutation=mutation)
    N = x.shape[0]
    Am = csr(A, pat, N)
    Mm = csr(M, pat, N)
    a1 = np.abs(Am @ np.ones(N)).max() / Am.diagonal().max()
    sym = max(abs(Am - Am.T).max(), abs(Mm - Mm.T).max())
    area = abs(M.sum() - 4 * np.pi) / (4 * np.pi)
    return a1, sym, area


def check_area_gradient(mutation=0, level=1, order=2):
    """d(1^T M 1)/dx = A X: the first variation of area is the stiffness matrix
    applied to the coordinates (exact for any rule, order, bulk or surface)."""
    x, e = meshes.icosphere(level, order)
    x = x * np.array([1.0, 0.9, 0.8])
    r = quadrature.default_rule(2, order)
    pat = oracle.pattern(e, x.shape[0])
    _, _, M, A, _ = oracle.assemble(x, e, 2, order, r.xi, r.w, pat=pat, mutation=mutation)
    gx, _ = oracle.adjoint(x, e, 2, order, r.xi, r.w, None, pat, gM=np.ones_like(M), mutation=mutation)
    AX = csr(A, pat, x.shape[0]) @ x
    return np.abs(gx - AX).max() / np.abs(AX).max()


def local_L(x, conn, d, p, rule, coef, elems, gM, gA, gC, pat, mutation=0):
    """Contribution of elements `elems` to L = gM.M + gA.A + gC.MC (for local FD)."""
    sub = conn[elems]
    M, A, C = oracle.local_matrices(x, sub, d, p, rule.xi, rule.w, None if coef is None else coef[elems],
                                    mutation=mutation)
    rp, ci = pat
    tot = 0.0
    for k, e in enumerate(elems):
        for a in range(sub.shape[1]):
            for b in range(sub.shape[1]):
                i, j = sub[k, a], sub[k, b]
                s = rp[i] + np.searchsorted(ci[rp[i]:rp[i + 1]], j)
                tot += gM[s] * M[k, a, b] + gA[s] * A[k, a, b] + gC[s] * C[k, a, b]
    return tot


def check_fd(mutation=0, n_coords=12, seed=7):
    """Central finite differences (h = 1e-6) of the local contributions to L
    against the adjoint, on a noisy P2 ellipsoid with a coefficient."""
    x, e = meshes.ellipsoid(1, sigma=1e-2, seed=seed)
    r = quadrature.tri_7pt_deg5()
    rng = np.random.default_rng(seed)
    coef = 1.0 + rng.random((e.shape[0], r.n_pts))
    pat = oracle.pattern(e, x.shape[0])
    nnz = pat[1].shape[0]
    # symmetric dL/d(values): derived from u^T M u + v^T A v + w^T MC w
    u, v, w = rng.normal(size=(3, x.shape[0]))
    rows = np.repeat(np.arange(x.shape[0]), np.diff(pat[0]))
    gM, gA, gC = u[rows] * u[pat[1]], v[rows] * v[pat[1]], w[rows] * w[pat[1]]
    gx, _ = oracle.adjoint(x, e, 2, 2, r.xi, r.w, coef, pat, gM, gA, gC, mutation=mutation)
    h = 1e-6
    worst = 0.0
    picks = rng.choice(x.shape[0] * 3, size=n_coords, replace=False)
    scale = np.abs(gx).max()
    for flat in picks:
        k, i = divmod(int(flat), 3)
        elems = np.nonzero((e == k).any(axis=1))[0]
        xp = x.copy()
        xp[k, i] += h
        xm = x.copy()
        xm[k, i] -= h
        fd = (local_L(xp, e, 2, 2, r, coef, elems, gM, gA, gC, pat, mutation) -
              local_L(xm, e, 2, 2, r, coef, elems, gM, gA, gC, pat, mutation)) / (2 * h)
        worst = max(worst, abs(fd - gx[k, i]) / scale)
    assert nnz > 0
    return worst


def check_load_is_mass_times_f(mutation=0):
    """The load vector of the interpolant f_h = sum f_i phi_i is b = M f (Sec. 2),
    on curved P2 surfaces, a P1 sphere, a P2 curve, P2 tets, and orders 3, 4 on
    the sphere and the cube; relative to max |b|."""
    worst = 0.0
    rng = np.random.default_rng(21)
    x1, t1 = meshes.kuhn_cube_p2(1, order=1)
    cases = [(meshes.icosphere(2, 2), 2, 2, None), (meshes.icosphere(2, 1), 2, 1, None),
             (meshes.closed_curve_p2(60, seed=4), 1, 2, None), (meshes.kuhn_cube_p2(2), 3, 2, None),
             (meshes.icosphere_high(1, 3), 2, 3, quadrature.tri_16pt_deg8()),
             (meshes.to_order(x1, t1, 4), 3, 4, quadrature.collapsed_gauss(3, 4))]
    for (x, e), d, p, r in cases:
        r = r or quadrature.default_rule(d, p)
        f = rng.standard_normal(x.shape[0])
        rp, ci, M, _, _ = oracle.assemble(x, e, d, p, r.xi, r.w, mutation=mutation)
        b = oracle.load(x, e, d, p, r.xi, r.w, f, mutation=mutation)
        Mf = csr(M, (rp, ci), x.shape[0]) @ f
        worst = max(worst, np.abs(b - Mf).max() / np.abs(Mf).max())
    return worst


def check_kll_identity_normal(mutation=0):
    """Non-linear vectors of Sec. 5.1 with the nodal 'normal' set to the node
    positions: nu_h is then the identity on Gamma_h, its tangential gradient is
    the tangential projector (Frobenius norm^2 = 2 exactly on a surface), so
    f1_k = 2 M x_k and f2 = 2 M H for any nodal H; a constant field gives 0."""
    worst = 0.0
    rng = np.random.default_rng(22)
    for order in (1, 2):
        x, e = meshes.ellipsoid(2, sigma=1e-2, seed=5) if order == 2 else meshes.icosphere(2, 1)
        r = quadrature.default_rule(2, order)
        H = rng.standard_normal(x.shape[0])
        u = np.column_stack([x, H])
        out = oracle.kll(x, e, order, r.xi, r.w, u, mutation=mutation)
        rp, ci, M, _, _ = oracle.assemble(x, e, 2, order, r.xi, r.w, mutation=mutation)
        Mm = csr(M, (rp, ci), x.shape[0])
        ref = np.vstack([2 * (Mm @ x[:, k]) for k in range(3)] + [2 * (Mm @ H)])
        worst = max(worst, np.abs(out - ref).max() / np.abs(ref).max())
        const = np.column_stack([np.tile([0.3, -0.2, 0.9], (x.shape[0], 1)), H])
        worst = max(worst, np.abs(oracle.kll(x, e, order, r.xi, r.w, const, mutation=mutation)).max())
    return worst


def check_mcf_sphere_step(mutation=0):
    """One step of Dziuk's scheme on the unit sphere shrinks it by the factor
    1 / (1 + 2 tau): with A x = M (2 x / r^2) for the sphere (H = 2 / r),
    (M + tau A) c x0 = M x0 gives c = 1 / (1 + 2 tau).  P2 icosphere level 3,
    tau = 1e-3: every node's radius against that factor."""
    x, e = meshes.icosphere(3, 2)
    r = quadrature.default_rule(2, 2)
    tau = 1e-3
    x1 = oracle.mcf_step(x, e, 2, 2, r.xi, r.w, tau, mutation=mutation)
    rad = np.linalg.norm(x1, axis=1)
    return float(np.abs(rad - 1.0 / (1.0 + 2.0 * tau)).max())


def check_adjoint_high_fd(mutation=0, seed=31):
    """Orders 3, 4: central differences (h = 1e-6) of L = gM.M + gA.A + gC.MC on
    a jittered P3 sphere against the adjoint, and dL/dc against the exact
    linearity of MC in the coefficient; relative to max |gradient|."""
    x, e = meshes.icosphere_high(0, 3)
    r = quadrature.tri_16pt_deg8()
    rng = np.random.default_rng(seed)
    x = x + rng.normal(0, 0.003, size=x.shape)
    coef = 1.0 + rng.random((e.shape[0], r.n_pts))
    pat = oracle.pattern(e, x.shape[0])
    gM, gA, gC = rng.normal(size=(3, pat[1].size))
    gx, gc = oracle.adjoint(x, e, 2, 3, r.xi, r.w, coef, pat, gM, gA, gC, mutation=mutation)
    h = 1e-6
    worst = 0.0
    scale = np.abs(gx).max()
    for flat in rng.choice(x.size, 6, replace=False):
        k, i = divmod(int(flat), 3)
        elems = np.nonzero((e == k).any(axis=1))[0]
        xp, xm = x.copy(), x.copy()
        xp[k, i] += h
        xm[k, i] -= h
        fd = (local_L(xp, e, 2, 3, r, coef, elems, gM, gA, gC, pat, mutation) -
              local_L(xm, e, 2, 3, r, coef, elems, gM, gA, gC, pat, mutation)) / (2 * h)
        worst = max(worst, abs(fd - gx[k, i]) / scale)
    for e0, q0 in ((0, 0), (e.shape[0] - 1, r.n_pts - 1)):
        cp, cm = coef.copy(), coef.copy()
        cp[e0, q0] += 0.5
        cm[e0, q0] -= 0.5
        dc = (local_L(x, e, 2, 3, r, cp, [e0], gM, gA, gC, pat, mutation) -
              local_L(x, e, 2, 3, r, cm, [e0], gM, gA, gC, pat, mutation))
        worst = max(worst, abs(dc - gc[e0, q0]) / np.abs(gc).max())
    return worst


ALL_CHECKS = {
    "lagrange": (check_lagrange, 1e-8),
    "affine_exact": (check_affine_exact, 1e-12),
    "p1_closed_forms": (check_p1_closed_forms, 1e-13),
    "half_disk": (check_half_disk, 1e-14),
    "area_gradient": (check_area_gradient, 1e-12),
    "fd": (check_fd, 1e-6),
    "load_is_mass_times_f": (check_load_is_mass_times_f, 1e-13),
    "kll_identity_normal": (check_kll_identity_normal, 1e-12),
    "mcf_sphere_step": (check_mcf_sphere_step, 2e-5),
    "adjoint_high_fd": (check_adjoint_high_fd, 1e-6),
}


def failing_checks(mutation):
    failed = []
    for name, (fn, tol) in ALL_CHECKS.items():
        try:
            val = fn(mutation=mutation)
        except Exception:  # a crash counts as a failed pin
            failed.append(name)
            continue
        if not np.isfinite(val) or val > tol:
            failed.append(name)
    return failed
